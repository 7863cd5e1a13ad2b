// EWA projection with SH colour (Sec. 3.1, Eq. 1) and its adjoint.
//
// One thread per Gaussian; attributes are read as coalesced SoA planes and
// the projected record is written as three 16-byte stores (AoS), the layout
// the tile compositor gathers by index.
#include "project.cuh"

namespace qn {
namespace {

template <int DEG>
__global__ void __launch_bounds__(256) k_project(int n, int S_, CamArgs cm, float blur, int tight,
                                                 const float *__restrict__ A, float4 *__restrict__ splat,
                                                 int4 *__restrict__ rects) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 s0, s1, s2;
    int4 rc;
    project_one<DEG>(cm, blur, tight, A, (size_t)S_, i, s0, s1, s2, rc);
    splat[3 * (size_t)i] = s0;
    splat[3 * (size_t)i + 1] = s1;
    splat[3 * (size_t)i + 2] = s2;
    rects[i] = rc;
}

template <int DEG>
__global__ void __launch_bounds__(128) k_project_bwd(int n, int S_, CamArgs cm, float blur,
                                                     const float *__restrict__ A,
                                                     const float4 *__restrict__ dsp,
                                                     const uint8_t *__restrict__ skip,
                                                     float *__restrict__ dA) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (skip && skip[i]) return;             // left untouched: the decode adjoint ignores skipped Gaussians
    project_bwd_one<DEG>(cm, blur, A, (size_t)S_, i, dsp, dA, (size_t)S_, i);
}

}  // namespace
}  // namespace qn

extern "C" int qn_project(int32_t n, int32_t n_stride, int32_t sh_degree, const float *attrs,
                          const qn_camera *cam_host, float blur, int32_t tight_rects, qn_splat *splats,
                          int32_t *rects, qn_stream_t stream) {
    qn::CamArgs cm;
    int st = qn::cam_args(cam_host, &cm);
    if (st) return st;
    QN_REQUIRE(n >= 0 && n_stride >= n && n_stride % 4 == 0, "bad n / n_stride");
    QN_REQUIRE(sh_degree >= 0 && sh_degree <= 3, "sh_degree must be 0..3 (got %d)", sh_degree);
    QN_REQUIRE(blur >= 0.f, "blur must be >= 0");
    QN_REQUIRE(n == 0 || (attrs && splats && rects), "null pointer argument");
    QN_REQUIRE(((uintptr_t)splats & 15) == 0 && ((uintptr_t)rects & 15) == 0, "splats/rects must be 16-byte aligned");
    if (n == 0) return QN_OK;
    decltype(&qn::k_project<0>) kern[4] = {qn::k_project<0>, qn::k_project<1>, qn::k_project<2>,
                                            qn::k_project<3>};
    kern[sh_degree]<<<qn::div_up(n, 256), 256, 0, qn::as_stream(stream)>>>(
        n, n_stride, cm, blur, tight_rects != 0, attrs, reinterpret_cast<float4 *>(splats),
        reinterpret_cast<int4 *>(rects));
    return qn::check_launch("qn_project");
}

extern "C" int qn_project_bwd(int32_t n, int32_t n_stride, int32_t sh_degree, const float *attrs,
                              const qn_camera *cam_host, float blur, const qn_splat *d_splats,
                              const uint8_t *skip, float *d_attrs, qn_stream_t stream) {
    qn::CamArgs cm;
    int st = qn::cam_args(cam_host, &cm);
    if (st) return st;
    QN_REQUIRE(n >= 0 && n_stride >= n && n_stride % 4 == 0, "bad n / n_stride");
    QN_REQUIRE(sh_degree >= 0 && sh_degree <= 3, "sh_degree must be 0..3 (got %d)", sh_degree);
    QN_REQUIRE(blur >= 0.f, "blur must be >= 0");
    QN_REQUIRE(n == 0 || (attrs && d_splats && d_attrs), "null pointer argument");
    QN_REQUIRE(((uintptr_t)d_splats & 15) == 0, "d_splats must be 16-byte aligned");
    if (n == 0) return QN_OK;
    decltype(&qn::k_project_bwd<0>) kern[4] = {qn::k_project_bwd<0>, qn::k_project_bwd<1>,
                                                qn::k_project_bwd<2>, qn::k_project_bwd<3>};
    kern[sh_degree]<<<qn::div_up(n, 128), 128, 0, qn::as_stream(stream)>>>(
        n, n_stride, cm, blur, attrs, reinterpret_cast<const float4 *>(d_splats), skip,
        d_attrs);
    return qn::check_launch("qn_project_bwd");
}
