// The compressed per-frame packet (Sec. 3.2.1 and App. B, storage): integer
// latents of every category flattened and entropy coded, decoders stored as
// bf16 bits, position residuals of the Gaussians whose gate is on in
// coordinate (COO) form, the gate binarised.
//
// Entropy coder: rANS (Duda's range asymmetric numeral systems, an arithmetic-
// coding variant) with a static model per category and frame -- frequencies
// quantised to M = 2^12, 32-bit state in [2^23, 2^31), byte renormalisation.
// A category's flattened vector (latent-major; symbol = integer latent + 128)
// is cut into streams of 8192 symbols, one GPU thread per stream: that is
// the parallelism the coder allows at a state per 8192 symbols (a state costs
// 4 bytes; fewer symbols per state would cost size, more would cost time).
//
// Packing: k_pack_symbols rounds the latents as the decode does and builds
// per-category histograms; the host quantises them into frequency tables;
// k_rans_encode codes every stream backwards into its own scratch slot;
// the host lays out the packet from the stream sizes and k_rans_compact,
// copies and k_coo_write fill it.  Unpacking: the host checks the header and
// uploads the packet; k_rans_decode writes float latents; k_coo_scatter
// rebuilds the position residuals with the gate forced to 0 or 1; the usual
// decode (qn_decode_residuals) then gives A_t.  A sender that carries forward
// its own unpacked packet and a receiver of the packet hold the same A_t bit
// for bit.
#include <cstring>
#include <vector>

#include "common.cuh"

namespace qn {
namespace {

constexpr int PK_STREAM = QN_PACKET_STREAM_SYMBOLS;
constexpr int PK_SCALE = QN_PACKET_SCALE_BITS, PK_M = 1 << PK_SCALE;
constexpr uint32_t PK_L = 1u << 23;
constexpr int PK_CAP = ((2 * PK_STREAM + 4) + 15) / 16 * 16;   // <= 2 bytes per symbol + the state
constexpr uint32_t PK_MAGIC = 0x46504E51u, PK_VERSION = 1;
constexpr int PK_THREADS = 128;

struct Tables {
    uint16_t f[QN_MAX_CATEGORIES][256];
    uint16_t c[QN_MAX_CATEGORIES][256];
};

struct CatInfo {
    int n_cat;
    int row[QN_MAX_CATEGORIES + 1];          // first latent row of each category
    int stream_begin[QN_MAX_CATEGORIES + 1]; // first stream of each category
    long long sym_off[QN_MAX_CATEGORIES];    // byte offset of each category's symbol vector
    long long len[QN_MAX_CATEGORIES];        // symbols of each category (lat_dim x n)
};

__device__ __forceinline__ int category_of_stream(const CatInfo &ci, int sid) {
    int c = 0;
#pragma unroll
    for (int k = 1; k < QN_MAX_CATEGORIES; ++k)
        if (k < ci.n_cat && sid >= ci.stream_begin[k]) c = k;
    return c;
}

// symbols of latent row r (category c) and per-category histograms
__global__ void __launch_bounds__(256) k_pack_symbols(int n, int S, const float *__restrict__ lat, CatInfo ci,
                                                      uint8_t *__restrict__ sym, unsigned *__restrict__ hist) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int r = blockIdx.y;
    int c = 0;
    for (int k = 1; k < ci.n_cat; ++k)
        if (r >= ci.row[k]) c = k;
    uint8_t *dst = sym + ci.sym_off[c] + (long long)(r - ci.row[c]) * n;
    for (int i = blockIdx.x * blockDim.x * 4 + threadIdx.x; i < n && i < (blockIdx.x + 1) * blockDim.x * 4;
         i += blockDim.x) {
        const float q = fminf(127.f, fmaxf(-128.f, rintf(lat[(size_t)r * S + i])));   // Eq. 5 rounding
        const int s = (int)q + 128;
        dst[i] = (uint8_t)s;
        atomicAdd(&h[s], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&hist[c * 256 + threadIdx.x], h[threadIdx.x]);
}

// One stream per thread, coded from its last symbol to its first into the
// end of its scratch slot: the final state (4 bytes, little-endian) then the
// renormalisation bytes in reverse order of emission.
__global__ void __launch_bounds__(PK_THREADS) k_rans_encode(int total, CatInfo ci, Tables tb,
                                                            const uint8_t *__restrict__ sym,
                                                            uint8_t *__restrict__ scratch,
                                                            unsigned *__restrict__ sizes) {
    const int sid = blockIdx.x * blockDim.x + threadIdx.x;
    if (sid >= total) return;
    const int c = category_of_stream(ci, sid);
    const long long j0 = (long long)(sid - ci.stream_begin[c]) * PK_STREAM;
    const int cnt = (int)min((long long)PK_STREAM, ci.len[c] - j0);
    const uint8_t *src = sym + ci.sym_off[c] + j0;
    uint8_t *end = scratch + (size_t)(sid + 1) * PK_CAP, *p = end;
    uint32_t x = PK_L;
    for (int k = cnt - 1; k >= 0; --k) {
        const int s = src[k];
        const uint32_t f = tb.f[c][s];
        const uint32_t x_max = ((PK_L >> PK_SCALE) << 8) * f;
        while (x >= x_max) {
            *--p = (uint8_t)(x & 0xFF);
            x >>= 8;
        }
        x = ((x / f) << PK_SCALE) + (x % f) + tb.c[c][s];
    }
    p -= 4;
    p[0] = (uint8_t)x;
    p[1] = (uint8_t)(x >> 8);
    p[2] = (uint8_t)(x >> 16);
    p[3] = (uint8_t)(x >> 24);
    sizes[sid] = (unsigned)(end - p);
}

// stream sid's bytes (the tail of its scratch slot) to packet + dst[sid]
__global__ void k_rans_compact(const uint8_t *__restrict__ scratch, const unsigned *__restrict__ sizes,
                               const unsigned long long *__restrict__ dst, uint8_t *__restrict__ packet) {
    const int sid = blockIdx.x;
    const unsigned sz = sizes[sid];
    const uint8_t *src = scratch + (size_t)(sid + 1) * PK_CAP - sz;
    uint8_t *out = packet + dst[sid];
    for (unsigned k = threadIdx.x; k < sz; k += blockDim.x) out[k] = src[k];
}

__global__ void k_gate_flags(int n, const float *__restrict__ gate, uint8_t *__restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flags[i] = gate[i] != 0.f;
}

// the COO section: n_coo, indices (increasing: the tail of the stable
// partition by gate != 0), then l_p [3][n_coo]
__global__ void k_coo_write(int n, int S, const int *__restrict__ perm, const int *__restrict__ n_first,
                            const float *__restrict__ lp, uint8_t *__restrict__ out) {
    const int nf = *n_first, n_coo = n - nf;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) *reinterpret_cast<unsigned *>(out) = (unsigned)n_coo;
    if (t >= n_coo) return;
    const int i = perm[nf + t];
    unsigned *idx = reinterpret_cast<unsigned *>(out + 4);
    float *val = reinterpret_cast<float *>(out + 4 + 4 * (size_t)n_coo);
    idx[t] = (unsigned)i;
#pragma unroll
    for (int d = 0; d < 3; ++d) val[(size_t)d * n_coo + t] = lp[(size_t)d * S + i];
}

struct DecodeStream {
    unsigned long long byte_off;   // within the uploaded packet
    unsigned bytes;
    int cat;
    long long j0;                  // first symbol within the category
    int count;
    int pad;
};

// Streams of one category per launch; the block builds the slot -> symbol
// table of the category in shared memory.  Writes lat[row + j / n][j % n] =
// symbol - 128.  A read past a stream's bytes sets *bad and stops.
__global__ void __launch_bounds__(PK_THREADS) k_rans_decode(int n, int S, int first, int count_streams,
                                                            const DecodeStream *__restrict__ ds,
                                                            const uint8_t *__restrict__ packet,
                                                            const uint16_t *__restrict__ freq, int row,
                                                            float *__restrict__ lat, int *__restrict__ bad) {
    __shared__ uint16_t f[256], cm[256];
    __shared__ uint8_t slot2sym[PK_M];
    for (int s = threadIdx.x; s < 256; s += blockDim.x) f[s] = freq[s];
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned acc = 0;
        for (int s = 0; s < 256; ++s) {
            cm[s] = (uint16_t)acc;
            acc += f[s];
        }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < 256; s += blockDim.x)
        for (int k = cm[s]; k < cm[s] + f[s] && k < PK_M; ++k) slot2sym[k] = (uint8_t)s;
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count_streams) return;
    const DecodeStream d = ds[first + t];
    const uint8_t *p = packet + d.byte_off, *end = p + d.bytes;
    if (d.bytes < 4) {
        atomicExch(bad, 1);
        return;
    }
    uint32_t x = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
    p += 4;
    for (int k = 0; k < d.count; ++k) {
        const uint32_t slot = x & (PK_M - 1);
        const int s = slot2sym[slot];
        x = (uint32_t)f[s] * (x >> PK_SCALE) + slot - cm[s];
        while (x < PK_L) {
            if (p >= end) {
                atomicExch(bad, 1);
                return;
            }
            x = (x << 8) | *p++;
        }
        const long long j = d.j0 + k;
        lat[(size_t)(row + j / n) * S + (j % n)] = (float)(s - 128);
    }
}

// position residuals and binarised gates from the COO section
__global__ void k_coo_scatter(int n, int S, int n_coo, const unsigned *__restrict__ idx,
                              const float *__restrict__ val, float *__restrict__ lp, float *__restrict__ la,
                              int *__restrict__ bad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_coo) return;
    const unsigned i = idx[t];
    if (i >= (unsigned)n || (t > 0 && idx[t - 1] >= i)) {
        atomicExch(bad, 1);
        return;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) lp[(size_t)d * S + i] = val[(size_t)d * n_coo + t];
    la[i] = 1e30f;
}

__global__ void k_fill(int n, float v, float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = v;
}

// ---------------------------------------------------------------- host side

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
size_t pad4(size_t v) { return (v + 3) & ~(size_t)3; }

// Quantised frequencies summing to M: f_s = max(1, floor(c_s M / T)) for
// c_s > 0; a shortfall goes to the most frequent symbol (the smallest such
// s), an excess is taken back in one pass over the symbols by decreasing f_s
// (then increasing s), each giving up to f_s - 1.
void normalize(const unsigned *counts, uint16_t *f_out) {
    unsigned long long total = 0;
    for (int s = 0; s < 256; ++s) total += counts[s];
    long long f[256];
    for (int s = 0; s < 256; ++s) f[s] = 0;
    if (total > 0) {
        long long sum = 0;
        for (int s = 0; s < 256; ++s) {
            if (counts[s] > 0) {
                const long long v = (long long)(((unsigned long long)counts[s] * PK_M) / total);
                f[s] = v > 1 ? v : 1;
            }
            sum += f[s];
        }
        long long d = PK_M - sum;
        if (d > 0) {
            int best = 0;
            for (int s = 1; s < 256; ++s)
                if (counts[s] > counts[best]) best = s;
            f[best] += d;
        } else if (d < 0) {
            int order[256];
            for (int s = 0; s < 256; ++s) order[s] = s;
            // stable insertion sort by decreasing f (ties keep increasing s)
            for (int a = 1; a < 256; ++a) {
                const int v = order[a];
                int b = a - 1;
                while (b >= 0 && f[order[b]] < f[v]) {
                    order[b + 1] = order[b];
                    --b;
                }
                order[b + 1] = v;
            }
            for (int k = 0; k < 256 && d < 0; ++k) {
                const int s = order[k];
                const long long t = (-d < f[s] - 1) ? -d : f[s] - 1;
                if (t > 0) {
                    f[s] -= t;
                    d += t;
                }
            }
        }
    }
    for (int s = 0; s < 256; ++s) f_out[s] = (uint16_t)f[s];
}

int layout_check(int n, const qn_decoder_layout *lay, CatInfo *ci, int *n_lat) {
    QN_REQUIRE(n >= 0, "n must be >= 0");
    QN_REQUIRE(lay, "layout is required");
    QN_REQUIRE(lay->n_cat >= 0 && lay->n_cat <= QN_MAX_CATEGORIES, "n_cat out of range");
    std::memset(ci, 0, sizeof(*ci));
    ci->n_cat = lay->n_cat;
    int row = 0, streams = 0;
    size_t off = 0;
    for (int c = 0; c < lay->n_cat; ++c) {
        QN_REQUIRE(lay->lat_dim[c] > 0 && lay->lat_dim[c] <= QN_MAX_LATENT && lay->attr_count[c] > 0,
                   "category %d: bad sizes", c);
        ci->row[c] = row;
        ci->stream_begin[c] = streams;
        ci->sym_off[c] = (long long)off;
        ci->len[c] = (long long)lay->lat_dim[c] * n;
        row += lay->lat_dim[c];
        streams += (int)((ci->len[c] + PK_STREAM - 1) / PK_STREAM);
        off += align256((size_t)ci->len[c]);
    }
    ci->row[lay->n_cat] = row;
    ci->stream_begin[lay->n_cat] = streams;
    *n_lat = row;
    return QN_OK;
}

struct PackWs {
    uint8_t *sym;
    unsigned *hist, *sizes;
    uint8_t *scratch;
    unsigned long long *dst;
    uint8_t *flags;
    int32_t *perm, *n_first;
    void *part;
    size_t part_bytes, total;
};

PackWs pack_ws(int n, const CatInfo &ci, void *base) {
    PackWs w;
    const int streams = ci.stream_begin[ci.n_cat];
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    size_t sym_bytes = 0;
    for (int c = 0; c < ci.n_cat; ++c) sym_bytes += align256((size_t)ci.len[c]);
    const size_t o_sym = take(sym_bytes), o_hist = take(sizeof(unsigned) * 256 * QN_MAX_CATEGORIES),
                 o_sizes = take(sizeof(unsigned) * (size_t)(streams + 1)),
                 o_scratch = take((size_t)PK_CAP * (size_t)streams),
                 o_dst = take(sizeof(unsigned long long) * (size_t)(streams + 1)), o_flags = take((size_t)n + 1),
                 o_perm = take(sizeof(int32_t) * ((size_t)n + 1)), o_nf = take(sizeof(int32_t));
    w.part_bytes = qn_partition_workspace_size(n);
    const size_t o_part = take(w.part_bytes);
    w.total = off;
    char *b = static_cast<char *>(base);
    w.sym = reinterpret_cast<uint8_t *>(b + o_sym);
    w.hist = reinterpret_cast<unsigned *>(b + o_hist);
    w.sizes = reinterpret_cast<unsigned *>(b + o_sizes);
    w.scratch = reinterpret_cast<uint8_t *>(b + o_scratch);
    w.dst = reinterpret_cast<unsigned long long *>(b + o_dst);
    w.flags = reinterpret_cast<uint8_t *>(b + o_flags);
    w.perm = reinterpret_cast<int32_t *>(b + o_perm);
    w.n_first = reinterpret_cast<int32_t *>(b + o_nf);
    w.part = b + o_part;
    return w;
}

size_t header_bytes(const CatInfo &ci) {
    return 24 + 16 * (size_t)ci.n_cat + 512 * (size_t)ci.n_cat + 4 * (size_t)ci.stream_begin[ci.n_cat];
}

void put32(std::vector<uint8_t> &v, uint32_t x) {
    for (int k = 0; k < 4; ++k) v.push_back((uint8_t)(x >> (8 * k)));
}

uint32_t get32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

}  // namespace
}  // namespace qn

extern "C" size_t qn_pack_workspace_size(int32_t n, const qn_decoder_layout *layout) {
    qn::CatInfo ci;
    int n_lat = 0;
    if (!layout || n < 0 || qn::layout_check(n, layout, &ci, &n_lat) != QN_OK) return 0;
    return qn::pack_ws(n, ci, nullptr).total;
}

extern "C" size_t qn_packet_max_bytes(int32_t n, const qn_decoder_layout *layout) {
    qn::CatInfo ci;
    int n_lat = 0;
    if (!layout || n < 0 || qn::layout_check(n, layout, &ci, &n_lat) != QN_OK) return 0;
    size_t b = qn::header_bytes(ci);
    for (int c = 0; c < ci.n_cat; ++c) {
        const int ns = ci.stream_begin[c + 1] - ci.stream_begin[c];
        b += qn::pad4(2 * (size_t)ci.len[c] + 4 * (size_t)ns);
        b += qn::pad4(2 * (size_t)layout->lat_dim[c] * layout->attr_count[c]);
    }
    return b + 4 + 16 * (size_t)n;
}

extern "C" int qn_pack_frame(int32_t n, int32_t n_stride, const qn_decoder_layout *layout, const float *lat,
                             const uint16_t *dec, const float *lp, const float *gate, void *workspace,
                             size_t workspace_bytes, uint8_t *packet, size_t packet_capacity, size_t *packet_bytes,
                             qn_stream_t stream) {
    qn::CatInfo ci;
    int n_lat = 0;
    const int rc = qn::layout_check(n, layout, &ci, &n_lat);
    if (rc != QN_OK) return rc;
    QN_REQUIRE(n_stride >= n, "n_stride must be >= n");
    QN_REQUIRE(workspace && packet && packet_bytes && (n == 0 || (lat && lp && gate)) &&
                   (ci.n_cat == 0 || dec),
               "null pointer argument");
    QN_REQUIRE(((uintptr_t)workspace & 255) == 0 && ((uintptr_t)packet & 3) == 0,
               "workspace must be 256-byte and packet 4-byte aligned");
    const qn::PackWs w = qn::pack_ws(n, ci, workspace);
    QN_REQUIRE(workspace_bytes >= w.total, "workspace too small (%zu < %zu)", workspace_bytes, w.total);
    cudaStream_t s = qn::as_stream(stream);
    const int streams = ci.stream_begin[ci.n_cat];
    auto cuda = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess) qn::set_error("qn_pack_frame: %s: %s", what, cudaGetErrorString(e));
        return e == cudaSuccess;
    };
    // symbols and histograms
    if (!cuda(cudaMemsetAsync(w.hist, 0, sizeof(unsigned) * 256 * QN_MAX_CATEGORIES, s), "memset")) return QN_ERR_CUDA;
    if (n > 0 && n_lat > 0) {
        qn::k_pack_symbols<<<dim3((unsigned)qn::div_up(n, 1024), (unsigned)n_lat), 256, 0, s>>>(n, n_stride, lat, ci,
                                                                                              w.sym, w.hist);
    }
    unsigned hist[QN_MAX_CATEGORIES * 256];
    if (!cuda(cudaMemcpyAsync(hist, w.hist, sizeof(hist), cudaMemcpyDeviceToHost, s), "histogram copy") ||
        !cuda(cudaStreamSynchronize(s), "synchronize"))
        return QN_ERR_CUDA;
    qn::Tables tb;
    std::memset(&tb, 0, sizeof(tb));
    for (int c = 0; c < ci.n_cat; ++c) {
        qn::normalize(hist + 256 * c, tb.f[c]);
        unsigned acc = 0;
        for (int k = 0; k < 256; ++k) {
            tb.c[c][k] = (uint16_t)acc;
            acc += tb.f[c][k];
        }
    }
    if (streams > 0)
        qn::k_rans_encode<<<qn::div_up(streams, qn::PK_THREADS), qn::PK_THREADS, 0, s>>>(streams, ci, tb, w.sym,
                                                                                        w.scratch, w.sizes);
    // COO indices: the Gaussians whose gate is not 0, in increasing order
    if (n > 0) {
        qn::k_gate_flags<<<qn::div_up(n, 256), 256, 0, s>>>(n, gate, w.flags);
        const int prc = qn_partition(n, w.flags, w.perm, w.n_first, w.part, w.part_bytes, stream);
        if (prc != QN_OK) return prc;
    } else if (!cuda(cudaMemsetAsync(w.n_first, 0, sizeof(int32_t), s), "memset")) {
        return QN_ERR_CUDA;
    }
    std::vector<unsigned> sizes((size_t)streams);
    int32_t n_first = 0;
    if ((streams > 0 &&
         !cuda(cudaMemcpyAsync(sizes.data(), w.sizes, sizeof(unsigned) * streams, cudaMemcpyDeviceToHost, s),
               "size copy")) ||
        !cuda(cudaMemcpyAsync(&n_first, w.n_first, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "count copy") ||
        !cuda(cudaStreamSynchronize(s), "synchronize"))
        return QN_ERR_CUDA;
    const int n_coo = n - n_first;
    // layout: header, payloads, decoders, COO
    std::vector<uint8_t> head;
    qn::put32(head, qn::PK_MAGIC);
    qn::put32(head, qn::PK_VERSION);
    qn::put32(head, (uint32_t)n);
    qn::put32(head, (uint32_t)ci.n_cat);
    qn::put32(head, (uint32_t)qn::PK_STREAM);
    qn::put32(head, (uint32_t)qn::PK_SCALE);
    std::vector<size_t> payload(ci.n_cat, 0);
    for (int c = 0; c < ci.n_cat; ++c) {
        for (int k = ci.stream_begin[c]; k < ci.stream_begin[c + 1]; ++k) payload[c] += sizes[k];
        qn::put32(head, (uint32_t)layout->lat_dim[c]);
        qn::put32(head, (uint32_t)layout->attr_count[c]);
        qn::put32(head, (uint32_t)(ci.stream_begin[c + 1] - ci.stream_begin[c]));
        qn::put32(head, (uint32_t)payload[c]);
    }
    for (int c = 0; c < ci.n_cat; ++c)
        for (int k = 0; k < 256; ++k) {
            head.push_back((uint8_t)tb.f[c][k]);
            head.push_back((uint8_t)(tb.f[c][k] >> 8));
        }
    for (int k = 0; k < streams; ++k) qn::put32(head, sizes[k]);
    std::vector<unsigned long long> dst((size_t)streams);
    size_t pos = head.size();
    for (int c = 0; c < ci.n_cat; ++c) {
        for (int k = ci.stream_begin[c]; k < ci.stream_begin[c + 1]; ++k) {
            dst[k] = pos;
            pos += sizes[k];
        }
        pos = qn::pad4(pos);
    }
    std::vector<size_t> dec_pos(ci.n_cat);
    size_t dec_src = 0;
    for (int c = 0; c < ci.n_cat; ++c) {
        dec_pos[c] = pos;
        pos += qn::pad4(2 * (size_t)layout->lat_dim[c] * layout->attr_count[c]);
    }
    const size_t coo_pos = pos;
    pos += 4 + 16 * (size_t)n_coo;
    QN_REQUIRE(pos <= packet_capacity, "packet capacity too small (%zu < %zu)", packet_capacity, pos);
    if (!cuda(cudaMemsetAsync(packet, 0, pos, s), "memset") ||
        !cuda(cudaMemcpyAsync(packet, head.data(), head.size(), cudaMemcpyHostToDevice, s), "header copy"))
        return QN_ERR_CUDA;
    if (streams > 0) {
        if (!cuda(cudaMemcpyAsync(w.dst, dst.data(), sizeof(unsigned long long) * streams, cudaMemcpyHostToDevice, s),
                  "offset copy"))
            return QN_ERR_CUDA;
        qn::k_rans_compact<<<streams, 256, 0, s>>>(w.scratch, w.sizes, w.dst, packet);
    }
    for (int c = 0; c < ci.n_cat; ++c) {
        const size_t bytes = 2 * (size_t)layout->lat_dim[c] * layout->attr_count[c];
        if (!cuda(cudaMemcpyAsync(packet + dec_pos[c], dec + dec_src / 2, bytes, cudaMemcpyDeviceToDevice, s),
                  "decoder copy"))
            return QN_ERR_CUDA;
        dec_src += bytes;
    }
    qn::k_coo_write<<<qn::div_up(n_coo > 0 ? n_coo : 1, 256), 256, 0, s>>>(n, n_stride, w.perm, w.n_first, lp,
                                                                           packet + coo_pos);
    *packet_bytes = pos;
    return qn::check_launch("qn_pack_frame");
}

extern "C" size_t qn_unpack_workspace_size(int32_t n, int32_t n_stride, const qn_decoder_layout *layout,
                                           size_t packet_bytes) {
    qn::CatInfo ci;
    int n_lat = 0;
    if (!layout || n < 0 || n_stride < n || qn::layout_check(n, layout, &ci, &n_lat) != QN_OK) return 0;
    size_t dec = 0;
    for (int c = 0; c < ci.n_cat; ++c) dec += 2 * (size_t)layout->lat_dim[c] * layout->attr_count[c];
    const int streams = ci.stream_begin[ci.n_cat];
    return qn::align256(packet_bytes) + qn::align256(sizeof(qn::DecodeStream) * (size_t)(streams + 1)) +
           qn::align256(sizeof(float) * (size_t)n_lat * n_stride) + qn::align256(dec + 4) +
           qn::align256(sizeof(float) * 3 * (size_t)n_stride) + qn::align256(sizeof(float) * ((size_t)n + 1)) +
           qn::align256(sizeof(int));
}

extern "C" int qn_unpack_frame(const uint8_t *packet_host, size_t packet_bytes, int32_t n, int32_t n_stride,
                               int32_t n_attr, const qn_decoder_layout *layout, const float *prev, float *out,
                               void *workspace, size_t workspace_bytes, qn_stream_t stream) {
    qn::CatInfo ci;
    int n_lat = 0;
    const int rc = qn::layout_check(n, layout, &ci, &n_lat);
    if (rc != QN_OK) return rc;
    QN_REQUIRE(n_stride >= n && n_stride % 4 == 0, "n_stride must be >= n and a multiple of 4");
    QN_REQUIRE(packet_host && prev && out && workspace, "null pointer argument");
    QN_REQUIRE(((uintptr_t)workspace & 255) == 0, "workspace must be 256-byte aligned");
    const size_t need = qn_unpack_workspace_size(n, n_stride, layout, packet_bytes);
    QN_REQUIRE(workspace_bytes >= need, "workspace too small (%zu < %zu)", workspace_bytes, need);
    // the header, checked against the layout and the size
    const uint8_t *h = packet_host;
    const int streams = ci.stream_begin[ci.n_cat];
    const size_t hb = qn::header_bytes(ci);
    QN_REQUIRE(packet_bytes >= hb, "corrupt packet: shorter than its header");
    QN_REQUIRE(qn::get32(h) == qn::PK_MAGIC && qn::get32(h + 4) == qn::PK_VERSION, "corrupt packet: bad magic");
    QN_REQUIRE(qn::get32(h + 8) == (uint32_t)n && qn::get32(h + 12) == (uint32_t)ci.n_cat &&
                   qn::get32(h + 16) == (uint32_t)qn::PK_STREAM && qn::get32(h + 20) == (uint32_t)qn::PK_SCALE,
               "packet does not match n / layout");
    std::vector<size_t> payload(ci.n_cat);
    for (int c = 0; c < ci.n_cat; ++c) {
        const uint8_t *m = h + 24 + 16 * c;
        QN_REQUIRE(qn::get32(m) == (uint32_t)layout->lat_dim[c] && qn::get32(m + 4) == (uint32_t)layout->attr_count[c] &&
                       qn::get32(m + 8) == (uint32_t)(ci.stream_begin[c + 1] - ci.stream_begin[c]),
                   "packet does not match the layout (category %d)", c);
        payload[c] = qn::get32(m + 12);
    }
    const uint8_t *ftab = h + 24 + 16 * ci.n_cat;
    for (int c = 0; c < ci.n_cat; ++c) {
        unsigned sum = 0;
        for (int k = 0; k < 256; ++k) sum += (unsigned)ftab[512 * c + 2 * k] | ((unsigned)ftab[512 * c + 2 * k + 1] << 8);
        QN_REQUIRE(sum == (unsigned)qn::PK_M || ci.len[c] == 0, "corrupt packet: frequency table %d", c);
    }
    const uint8_t *stab = ftab + 512 * ci.n_cat;
    std::vector<qn::DecodeStream> ds((size_t)streams + 1);
    size_t pos = hb;
    for (int c = 0; c < ci.n_cat; ++c) {
        size_t sum = 0;
        for (int k = ci.stream_begin[c]; k < ci.stream_begin[c + 1]; ++k) {
            const unsigned sz = qn::get32(stab + 4 * k);
            const long long j0 = (long long)(k - ci.stream_begin[c]) * qn::PK_STREAM;
            ds[k] = {pos + sum, sz, c, j0, (int)std::min<long long>(qn::PK_STREAM, ci.len[c] - j0), 0};
            sum += sz;
        }
        QN_REQUIRE(sum == payload[c], "corrupt packet: stream sizes of category %d", c);
        pos = qn::pad4(pos + sum);
    }
    std::vector<size_t> dec_pos(ci.n_cat);
    size_t dec_total = 0;
    for (int c = 0; c < ci.n_cat; ++c) {
        dec_pos[c] = pos;
        const size_t b = 2 * (size_t)layout->lat_dim[c] * layout->attr_count[c];
        dec_total += b;
        pos += qn::pad4(b);
    }
    QN_REQUIRE(pos + 4 <= packet_bytes, "corrupt packet: truncated");
    const uint32_t n_coo = qn::get32(h + pos);
    QN_REQUIRE(n_coo <= (uint32_t)n && pos + 4 + 16 * (size_t)n_coo == packet_bytes,
               "corrupt packet: COO section size");
    const size_t coo_pos = pos;
    // device workspace
    char *b = static_cast<char *>(workspace);
    uint8_t *pk = reinterpret_cast<uint8_t *>(b);
    b += qn::align256(packet_bytes);
    qn::DecodeStream *d_ds = reinterpret_cast<qn::DecodeStream *>(b);
    b += qn::align256(sizeof(qn::DecodeStream) * (size_t)(streams + 1));
    float *lat = reinterpret_cast<float *>(b);
    b += qn::align256(sizeof(float) * (size_t)n_lat * n_stride);
    uint16_t *dec = reinterpret_cast<uint16_t *>(b);
    b += qn::align256(dec_total + 4);
    float *lp = reinterpret_cast<float *>(b);
    b += qn::align256(sizeof(float) * 3 * (size_t)n_stride);
    float *la = reinterpret_cast<float *>(b);
    b += qn::align256(sizeof(float) * ((size_t)n + 1));
    int *bad = reinterpret_cast<int *>(b);
    cudaStream_t s = qn::as_stream(stream);
    auto cuda = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess) qn::set_error("qn_unpack_frame: %s: %s", what, cudaGetErrorString(e));
        return e == cudaSuccess;
    };
    if (!cuda(cudaMemcpyAsync(pk, packet_host, packet_bytes, cudaMemcpyHostToDevice, s), "packet copy") ||
        (streams > 0 && !cuda(cudaMemcpyAsync(d_ds, ds.data(), sizeof(qn::DecodeStream) * streams,
                                              cudaMemcpyHostToDevice, s),
                              "stream table copy")) ||
        !cuda(cudaMemsetAsync(bad, 0, sizeof(int), s), "memset") ||
        !cuda(cudaMemsetAsync(lp, 0, sizeof(float) * 3 * (size_t)n_stride, s), "memset"))
        return QN_ERR_CUDA;
    for (int c = 0; c < ci.n_cat; ++c) {
        const int first = ci.stream_begin[c], cnt = ci.stream_begin[c + 1] - first;
        if (cnt > 0)
            qn::k_rans_decode<<<qn::div_up(cnt, qn::PK_THREADS), qn::PK_THREADS, 0, s>>>(
                n, n_stride, first, cnt, d_ds, pk, reinterpret_cast<const uint16_t *>(pk + (ftab - h) + 512 * c),
                ci.row[c], lat, bad);
    }
    size_t dec_off = 0;
    for (int c = 0; c < ci.n_cat; ++c) {
        const size_t bytes = 2 * (size_t)layout->lat_dim[c] * layout->attr_count[c];
        if (!cuda(cudaMemcpyAsync(reinterpret_cast<uint8_t *>(dec) + dec_off, pk + dec_pos[c], bytes,
                                  cudaMemcpyDeviceToDevice, s),
                  "decoder copy"))
            return QN_ERR_CUDA;
        dec_off += bytes;
    }
    if (n > 0) qn::k_fill<<<qn::div_up(n, 256), 256, 0, s>>>(n, -1e30f, la);
    if (n_coo > 0)
        qn::k_coo_scatter<<<qn::div_up(n_coo, 256), 256, 0, s>>>(
            n, n_stride, (int)n_coo, reinterpret_cast<const unsigned *>(pk + coo_pos + 4),
            reinterpret_cast<const float *>(pk + coo_pos + 4 + 4 * (size_t)n_coo), lp, la, bad);
    int launch = qn::check_launch("qn_unpack_frame");
    if (launch != QN_OK) return launch;
    // the gate forced to exactly 0 or 1: sigmoid(+-1e30) is 1 or 0 and the
    // stretched value lands outside [0, 1] on both sides
    const qn_gate_params bin = {1.f, -0.5f, 1.5f};
    const int drc = qn_decode_residuals(n, n_stride, n_attr, prev, lat, dec, layout, lp, la, &bin, nullptr, out,
                                        nullptr, nullptr, stream);
    if (drc != QN_OK) return drc;
    int bad_host = 0;
    if (!cuda(cudaMemcpyAsync(&bad_host, bad, sizeof(int), cudaMemcpyDeviceToHost, s), "flag copy") ||
        !cuda(cudaStreamSynchronize(s), "synchronize"))
        return QN_ERR_CUDA;
    QN_REQUIRE(!bad_host, "corrupt packet: stream or COO data out of range");
    return QN_OK;
}
