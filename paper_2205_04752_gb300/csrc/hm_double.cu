// hm_double.cu -- the double-layer operator K_h of Section 4.2, Eq. (Kh), in
// collocation form (rows 3i + a at the triangles' centroids, columns 3p + b
// for the hat function of vertex p and component b):
//
//   K_h = diag(K_Delta) - diag(V_Delta) T_h + E/(1+nu) V_h T_h.
//
// K_Delta (the Laplace double layer weighted by the hat functions) is its own
// H-matrix on the partition triangles x vertices (hm_build_vertex_tree,
// assembled by hm_aca_assemble; applied by the evaluation operator's passes
// with c1 = 1, c2 = 0).  T_h, the surface curls T_kl = n_l d_k - n_k d_l of
// the hat functions, is constant on each flat triangle and is applied here
// triangle by triangle.  With V_h = c1 diag(V_Delta) + c2 [V_kl] the last two
// terms are one single-layer product with the coefficients
//   c1' = E c1 / (1+nu) - 1 = (1 - 2nu) / (2 (1 - nu)),
//   c2' = E c2 / (1+nu)     = 1 / (2 (1 - nu)),
// so K_h u = (K_Delta x I) u + V_h[c1', c2'] (T_h u), E cancelling.
#include <algorithm>
#include <cmath>

#include "hm_internal.h"

namespace hm {
namespace {

// w = T_h u for every triangle (cluster position p, original id rperm[p]):
//   w_a = sum over the corners c of [ g_c,a (n . u_c) - n_a (g_c . u_c) ],
// g_c = n x (v_{c+2} - v_{c+1}) / (twice the area), the gradient of the hat
// function of corner c on the triangle; u (3 per vertex) and w (3 per
// triangle) in the original orders.
__global__ void dl_curl_kernel(int64_t M, const int32_t* __restrict__ rperm, const double* __restrict__ tri,
                               const double* __restrict__ nrm, const int32_t* __restrict__ T,
                               const double* __restrict__ u, double* __restrict__ w)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    const int64_t t = rperm[p];
    const double* v = tri + 9 * p;
    const double n[3] = {nrm[4 * p], nrm[4 * p + 1], nrm[4 * p + 2]};
    const double a2 = nrm[4 * p + 3];
    double o[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double* q1 = v + 3 * ((c + 1) % 3);
        const double* q2 = v + 3 * ((c + 2) % 3);
        const double e[3] = {q2[0] - q1[0], q2[1] - q1[1], q2[2] - q1[2]};
        const double g[3] = {(n[1] * e[2] - n[2] * e[1]) / a2, (n[2] * e[0] - n[0] * e[2]) / a2,
                             (n[0] * e[1] - n[1] * e[0]) / a2};
        const double* uc = u + 3 * (int64_t)T[3 * t + c];
        const double nu_ = n[0] * uc[0] + n[1] * uc[1] + n[2] * uc[2];
        const double gu = g[0] * uc[0] + g[1] * uc[1] + g[2] * uc[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) o[a] += g[a] * nu_ - n[a] * gu;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) w[3 * t + a] = o[a];
}

}  // namespace
}  // namespace hm

using namespace hm;

extern "C" int hm_double_layer_matvec(hm_matrix* V, const hm_matrix* K, const double* u, double* y, int32_t nrhs,
                                      int32_t form, void* stream)
{
    if (!V || !K || !u || !y) return fail(HM_EINVAL, "hm_double_layer_matvec: NULL argument");
    if (V->rect) return fail(HM_EINVAL, "hm_double_layer_matvec: V must be the single layer (a triangle tree's matrix)");
    if (!K->dl) return fail(HM_EINVAL, "hm_double_layer_matvec: K must be the double layer's K_Delta (a vertex tree's matrix)");
    if (K->mesh_fp != V->mesh_fp || K->Mr != V->M)
        return fail(HM_EINVAL, "hm_double_layer_matvec: V and K were built on different meshes");
    if (nrhs < 1) return fail(HM_EINVAL, "hm_double_layer_matvec: nrhs %d < 1", nrhs);
    if (form < HM_FP64 || form >= HM_NFORMS) return fail(HM_EINVAL, "hm_double_layer_matvec: unknown form %d", form);
    if (!V->packed[form]) return fail(HM_EINVAL, "hm_double_layer_matvec: form %d of V not packed (hm_pack)", form);
    if (K->aca_deferred || K->compacted || !K->U64.p)
        return fail(HM_EINVAL, "hm_double_layer_matvec: K has no assembled FP64 factors");
    const int64_t M = V->M, nv = K->M;
    const char* ub = (const char*)u;
    const char* yb = (const char*)y;
    const size_t us = (size_t)nrhs * 3 * nv * 8, ys = (size_t)nrhs * 3 * M * 8;
    if (ub < yb + ys && yb < ub + us) return fail(HM_EINVAL, "hm_double_layer_matvec: u and y overlap");
    cudaStream_t s = (cudaStream_t)stream;
    const double nu = V->nu;
    const double c1 = (1.0 - 2.0 * nu) / (2.0 * (1.0 - nu)), c2 = 1.0 / (2.0 * (1.0 - nu));
    for (int32_t r = 0; r < nrhs; ++r) {
        const double* ur = u + (size_t)r * 3 * nv;
        double* yr = y + (size_t)r * 3 * M;
        dl_curl_kernel<<<(unsigned)((M + 127) / 128), 128, 0, s>>>(M, K->d_rperm.as<int32_t>(), K->g_tri.as<double>(),
                                                                  K->g_nrm.as<double>(), K->d_tris.as<int32_t>(), ur,
                                                                  K->dl_w.as<double>());
        HM_CUDA(cudaGetLastError());
        int rc = matvec_device_coeffs(*V, K->dl_w.as<double>(), yr, form, c1, c2, s);
        if (rc) return rc;
        if ((rc = eval_apply(*K, ur, yr, 1, HM_FP64, true, s))) return rc;
    }
    return HM_OK;
}
