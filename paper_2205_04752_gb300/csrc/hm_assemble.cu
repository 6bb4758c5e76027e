// hm_assemble.cu -- device assembly of the collocation Lame single-layer
// H-matrix: quadrature points, near-field blocks computed entry by entry, and
// batched ACA (Algorithm 1) over all admissible blocks and scalar kernels.
//
// Quadrature contract (the paper names no rule):
//   * self pair: tau split at its centroid into three sub-triangles; Duffy
//     map collapsing the apex, exact radial integral, 32 Gauss-Legendre
//     points for the remaining 1-D integral per sub-triangle;
//   * other pairs: Radon's 7-point degree-5 rule, on tau_j itself when
//     |x - g_j|^2 >= 4 diam(tau_j)^2, otherwise on the leaves of a recursive
//     4-way midpoint subdivision (same test per sub-triangle, depth < 8).
// The subdivision decisions are taken with separately rounded operations
// (no FMA) so that they do not depend on instruction selection.
//
// Scalar kernels, index kern: 0 V_Delta (1/r), 1 V_11, 2 V_12, 3 V_13, 4 V_22,
// 5 V_23, 6 V_33 (d_k d_l / r^3, d = x - y), each with the factor 1/(4 pi)
// (Eq. (Vh), prefactor read as 1/(4 pi)).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "hm_internal.h"

namespace hm {
namespace {

constexpr int kGL = 32;         // Gauss-Legendre points of the self term
constexpr int kMaxDepth = 8;    // subdivision depth cap
constexpr int kStack = 3 * kMaxDepth + 1;
constexpr int kAcaThreads = 256;
constexpr int kAcaWarps = kAcaThreads / 32;
constexpr int kKmaxLimit = 256;
constexpr double kInv4Pi = 0.07957747154594767;  // 1 / (4 pi)
constexpr double kAcaDelta = 1e-14;  // "v~ vanishes": max|v~| <= delta max|raw row|
constexpr double kAcaTie = 1e-10;    // argmax ties: smallest index within this relative gap

__constant__ double c_lam[21];  // Radon 7-point barycentric nodes
__constant__ double c_w7[7];    // and weights (sum 1)
__constant__ double c_glx[kGL]; // Gauss-Legendre nodes / weights on [0, 1]
__constant__ double c_glw[kGL];

struct Geom {
    const double* coll;   // M x 3, cluster order: collocation points (centroids)
    const double* tri;    // M x 9: vertices
    const double* qp;     // M x 21: 7-point nodes
    const double* qw;     // M x 7: weights * area / (4 pi)
    const double* diam2;  // M: max squared edge length
    const double* xr;     // rows: coll, or the points of the evaluation operator (cluster order)
    int square;           // rows are the collocation points: (i, i) is a self pair
    // the double layer's K_Delta (columns: hat functions of the vertices)
    const double* nrm = nullptr;        // M x 4: unit normal, twice the area
    const int32_t* star_ptr = nullptr;  // vertex cluster position -> its star entries
    const int32_t* star = nullptr;      // triangle position * 4 + local index of the vertex
};

// ---------------------------------------------------------------- host tables
// Radon's rule (Stroud T2:5-1): centroid weight 9/40; nodes (a, a, 1-2a) with
// a = (6 -+ sqrt 15)/21 and weights (155 -+ sqrt 15)/1200.
void radon_table(double lam[21], double w[7])
{
    const double r15 = std::sqrt(15.0);
    const double a[2] = {(6.0 - r15) / 21.0, (6.0 + r15) / 21.0};
    const double wt[2] = {(155.0 - r15) / 1200.0, (155.0 + r15) / 1200.0};
    lam[0] = lam[1] = lam[2] = 1.0 / 3.0;
    w[0] = 9.0 / 40.0;
    int q = 1;
    for (int g = 0; g < 2; ++g) {
        const double b = 1.0 - 2.0 * a[g];
        const double pts[3][3] = {{a[g], a[g], b}, {a[g], b, a[g]}, {b, a[g], a[g]}};
        for (int p = 0; p < 3; ++p, ++q) {
            for (int c = 0; c < 3; ++c) lam[3 * q + c] = pts[p][c];
            w[q] = wt[g];
        }
    }
}

// Gauss-Legendre on [0,1] from the Golub-Welsch view: Newton iteration on the
// Legendre recurrence from Chebyshev-like starting points.
void gauss_legendre_table(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double t = std::cos(M_PI * (n - i - 0.25) / (n + 0.5));  // ascending roots
        double pn = 0.0, pn1 = 0.0;
        for (int it = 0; it < 60; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            pn = p1;
            pn1 = p0;
            double d = n * (pn1 - t * pn) / (1.0 - t * t);
            double step = pn / d;
            t -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double d = n * (p0 - t * p1) / (1.0 - t * t);
        x[i] = 0.5 * (1.0 + t);
        w[i] = 1.0 / ((1.0 - t * t) * d * d);  // = 0.5 * 2 / ((1-t^2) P_n'^2)
    }
}

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ double sq_dist_rn(const double* a, const double* b)
{
    double d0 = __dsub_rn(a[0], b[0]), d1 = __dsub_rn(a[1], b[1]), d2 = __dsub_rn(a[2], b[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
}

// x is close to the (sub-)triangle v[0..8] when |x - g|^2 < 4 diam^2
__device__ __forceinline__ bool is_near_rn(const double* x, const double* v)
{
    double g[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) g[k] = __ddiv_rn(__dadd_rn(__dadd_rn(v[k], v[3 + k]), v[6 + k]), 3.0);
    double e0 = sq_dist_rn(v, v + 3), e1 = sq_dist_rn(v + 3, v + 6), e2 = sq_dist_rn(v + 6, v);
    double dm = fmax(fmax(e0, e1), e2);
    return sq_dist_rn(x, g) < __dmul_rn(4.0, dm);
}

// accumulate the seven kernels of one source point with weight w (d = x - y)
__device__ __forceinline__ void point7(double d0, double d1, double d2, double w, double* acc)
{
    double r2 = d0 * d0 + d1 * d1 + d2 * d2;
    double ir = rsqrt(r2);
    double wir = w * ir;
    double wir3 = wir * ir * ir;
    acc[0] += wir;
    acc[1] += wir3 * d0 * d0;
    acc[2] += wir3 * d0 * d1;
    acc[3] += wir3 * d0 * d2;
    acc[4] += wir3 * d1 * d1;
    acc[5] += wir3 * d1 * d2;
    acc[6] += wir3 * d2 * d2;
}

// 7-point rule on one (sub-)triangle v, all kernels, weights include area
__device__ void rule7_all(const double* x, const double* v, double* acc)
{
    double u[3], w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        u[k] = v[3 + k] - v[k];
        w[k] = v[6 + k] - v[k];
    }
    double n0 = u[1] * w[2] - u[2] * w[1], n1 = u[2] * w[0] - u[0] * w[2],
           n2 = u[0] * w[1] - u[1] * w[0];
    double area = 0.5 * sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        double y[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            y[k] = c_lam[3 * q] * v[k] + c_lam[3 * q + 1] * v[3 + k] + c_lam[3 * q + 2] * v[6 + k];
        point7(x[0] - y[0], x[1] - y[1], x[2] - y[2], c_w7[q], s);
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) acc[c] += area * s[c];
}

// adaptive rule for a point outside triangle v: depth-first over the midpoint
// subdivision (children: corner 0, corner 1, corner 2, middle); returns the
// number of leaves the 7-point rule was applied on
__device__ int adaptive7(const double* x, const double* v0, double* acc)
{
    int leaves = 0;
    double st[kStack][9];
    int dep[kStack];
    int top = 0;
#pragma unroll
    for (int c = 0; c < 9; ++c) st[0][c] = v0[c];
    dep[0] = 0;
    top = 1;
    while (top > 0) {
        --top;
        double v[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) v[c] = st[top][c];
        int d = dep[top];
        if (d < kMaxDepth && is_near_rn(x, v)) {
            double ab[3], bc[3], ca[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ab[k] = __dmul_rn(__dadd_rn(v[k], v[3 + k]), 0.5);
                bc[k] = __dmul_rn(__dadd_rn(v[3 + k], v[6 + k]), 0.5);
                ca[k] = __dmul_rn(__dadd_rn(v[6 + k], v[k]), 0.5);
            }
            // push in reverse so that the pop order is corner 0, 1, 2, middle
            const double* kids[4][3] = {{ab, bc, ca}, {ca, bc, v + 6}, {ab, v + 3, bc}, {v, ab, ca}};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int k = 0; k < 3; ++k) st[top][3 * p + k] = kids[q][p][k];
                dep[top] = d + 1;
                ++top;
            }
        } else {
            rule7_all(x, v, acc);
            ++leaves;
        }
    }
    return leaves;
}

// self pair: x is the centroid of v; Duffy map per edge sub-triangle
__device__ void self7(const double* x, const double* v, double* acc)
{
#pragma unroll 1
    for (int e = 0; e < 3; ++e) {
        const double* pa = v + 3 * e;
        const double* pb = v + 3 * ((e + 1) % 3);
        double a[3], b[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            a[k] = pa[k] - x[k];
            b[k] = pb[k] - pa[k];
        }
        double n0 = a[1] * b[2] - a[2] * b[1], n1 = a[2] * b[0] - a[0] * b[2],
               n2 = a[0] * b[1] - a[1] * b[0];
        double cr = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
#pragma unroll 4
        for (int q = 0; q < kGL; ++q) {
            double t = c_glx[q];
            point7(a[0] + t * b[0], a[1] + t * b[1], a[2] + t * b[2], c_glw[q] * cr, acc);
        }
    }
}

// all seven kernels of pair (i, j) (row and column cluster positions), times
// 1/(4 pi).  Returns the rule taken: -1 the self term, 0 the 7-point rule on
// the whole triangle, n > 0 the 7-point rule on n subdivision leaves.
__device__ int entry7(const Geom& g, int i, int j, double* acc)
{
#pragma unroll
    for (int c = 0; c < 7; ++c) acc[c] = 0.0;
    const double* x = g.xr + 3 * (size_t)i;
    const double* v = g.tri + 9 * (size_t)j;
    int rule;
    if (g.square && i == j) {
        self7(x, v, acc);
        rule = -1;
    } else if (sq_dist_rn(x, g.coll + 3 * (size_t)j) < __dmul_rn(4.0, g.diam2[j])) {
        rule = adaptive7(x, v, acc);
    } else {
        const double* qp = g.qp + 21 * (size_t)j;
        const double* qw = g.qw + 7 * (size_t)j;
#pragma unroll
        for (int q = 0; q < 7; ++q)
            point7(x[0] - qp[3 * q], x[1] - qp[3 * q + 1], x[2] - qp[3 * q + 2], qw[q], acc);
        return 0;  // qw already holds 1/(4 pi)
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) acc[c] *= kInv4Pi;
    return rule;
}

// one scalar kernel of pair (i, j): the far (7-point) path is specialised
__device__ __forceinline__ double entry1(const Geom& g, int i, int j, int kern, int ka, int kb)
{
    const double* x = g.xr + 3 * (size_t)i;
    if (!(g.square && i == j) && !(sq_dist_rn(x, g.coll + 3 * (size_t)j) < __dmul_rn(4.0, g.diam2[j]))) {
        const double* qp = g.qp + 21 * (size_t)j;
        const double* qw = g.qw + 7 * (size_t)j;
        double x0 = x[0], x1 = x[1], x2 = x[2];
        double acc = 0.0;
        if (kern == 0) {
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                double d0 = x0 - qp[3 * q], d1 = x1 - qp[3 * q + 1], d2 = x2 - qp[3 * q + 2];
                acc += qw[q] * rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                double d0 = x0 - qp[3 * q], d1 = x1 - qp[3 * q + 1], d2 = x2 - qp[3 * q + 2];
                double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                double ir = rsqrt(r2);
                double da = ka == 0 ? d0 : (ka == 1 ? d1 : d2);
                double db = kb == 0 ? d0 : (kb == 1 ? d1 : d2);
                acc += qw[q] * ir * ir * ir * (da * db);
            }
        }
        return acc;
    }
    double a7[7];
    entry7(g, i, j, a7);
    return a7[kern];
}

// ---------------------------------------------------------------- double layer
// K_Delta of Eq. (Kh) in collocation form: entry (i, p) is
//   1/(4 pi) sum over the triangles tau_j holding vertex p of
//   int_{tau_j} (c_i - y).n_j / |c_i - y|^3 psi_p(y) ds_y,
// psi_p the hat function of p, which on tau_j is the barycentric coordinate
// of p's corner; the collocation point's own flat panel gives 0.  The same
// quadrature contract as the single layer: the 7-point rule on tau_j, or on
// the leaves of its midpoint subdivision when c_i is near.

// the 7-point rule on sub-triangle s of triangle v (normal nr[0..2], twice
// its area nr[3]) for the corner a of v: area(s) sum_q w_q k(x - y_q) lambda_a(y_q)
__device__ double dl_rule7(const double* x, const double* s, const double* v, const double* nr, int a)
{
    double u[3], w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        u[k] = s[3 + k] - s[k];
        w[k] = s[6 + k] - s[k];
    }
    const double n0 = u[1] * w[2] - u[2] * w[1], n1 = u[2] * w[0] - u[0] * w[2], n2 = u[0] * w[1] - u[1] * w[0];
    const double area = 0.5 * sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    const double* q1 = v + 3 * ((a + 1) % 3);
    const double* q2 = v + 3 * ((a + 2) % 3);
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        double y[3], d[3], e1[3], e2[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            y[k] = c_lam[3 * q] * s[k] + c_lam[3 * q + 1] * s[3 + k] + c_lam[3 * q + 2] * s[6 + k];
            d[k] = x[k] - y[k];
            e1[k] = q1[k] - y[k];
            e2[k] = q2[k] - y[k];
        }
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double r = sqrt(r2);
        const double kv = (d[0] * nr[0] + d[1] * nr[1] + d[2] * nr[2]) / (r2 * r);
        const double c0 = e1[1] * e2[2] - e1[2] * e2[1], c1 = e1[2] * e2[0] - e1[0] * e2[2],
                     c2 = e1[0] * e2[1] - e1[1] * e2[0];
        const double lam = (c0 * nr[0] + c1 * nr[1] + c2 * nr[2]) / nr[3];
        acc += c_w7[q] * kv * lam;
    }
    return area * acc;
}

// the subdivision of adaptive7 (same test, same order) with the double-layer
// integrand for corner a of v
__device__ double dl_adaptive(const double* x, const double* v0, const double* nr, int a)
{
    double st[kStack][9];
    int dep[kStack];
#pragma unroll
    for (int c = 0; c < 9; ++c) st[0][c] = v0[c];
    dep[0] = 0;
    int top = 1;
    double acc = 0.0;
    while (top > 0) {
        --top;
        double v[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) v[c] = st[top][c];
        const int d = dep[top];
        if (d < kMaxDepth && is_near_rn(x, v)) {
            double ab[3], bc[3], ca[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ab[k] = __dmul_rn(__dadd_rn(v[k], v[3 + k]), 0.5);
                bc[k] = __dmul_rn(__dadd_rn(v[3 + k], v[6 + k]), 0.5);
                ca[k] = __dmul_rn(__dadd_rn(v[6 + k], v[k]), 0.5);
            }
            const double* kids[4][3] = {{ab, bc, ca}, {ca, bc, v + 6}, {ab, v + 3, bc}, {v, ab, ca}};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int k = 0; k < 3; ++k) st[top][3 * p + k] = kids[q][p][k];
                dep[top] = d + 1;
                ++top;
            }
        } else {
            acc += dl_rule7(x, v, v0, nr, a);
        }
    }
    return acc;
}

// corner a of triangle j (cluster position) at point x, times 1/(4 pi)
__device__ double dl_pair(const Geom& g, const double* x, int j, int a)
{
    if (sq_dist_rn(x, g.coll + 3 * (size_t)j) < __dmul_rn(4.0, g.diam2[j]))
        return dl_adaptive(x, g.tri + 9 * (size_t)j, g.nrm + 4 * (size_t)j, a) * kInv4Pi;
    // far: the rule's nodes and weights (area / (4 pi) folded in) of the
    // geometry tables; lambda_a at node q is the rule's own coordinate
    const double* qp = g.qp + 21 * (size_t)j;
    const double* qw = g.qw + 7 * (size_t)j;
    const double* nr = g.nrm + 4 * (size_t)j;
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const double d0 = x[0] - qp[3 * q], d1 = x[1] - qp[3 * q + 1], d2 = x[2] - qp[3 * q + 2];
        const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
        const double r = sqrt(r2);
        acc += qw[q] * ((d0 * nr[0] + d1 * nr[1] + d2 * nr[2]) / (r2 * r)) * c_lam[3 * q + a];
    }
    return acc;
}

// K_Delta (i, p): row i (triangle position), column p (vertex position)
__device__ double dl_entry(const Geom& g, int i, int p)
{
    const double* x = g.xr + 3 * (size_t)i;
    double acc = 0.0;
    for (int e = g.star_ptr[p]; e < g.star_ptr[p + 1]; ++e) {
        const int sj = g.star[e], j = sj >> 2, a = sj & 3;
        if (j != i) acc += dl_pair(g, x, j, a);
    }
    return acc;
}

// near blocks of K_Delta: one CTA per block; stored as the six values of the
// single layer's layout with K_Delta in the first and zeros elsewhere (the
// product's trace is then K_Delta itself)
__global__ void __launch_bounds__(128) dl_near_kernel(Geom g, const Blk* __restrict__ blks,
                                                      const int64_t* __restrict__ noff, double* __restrict__ N)
{
    Blk b = blks[blockIdx.x];
    double* out = N + noff[blockIdx.x];
    const int pairs = b.m * b.n;
    for (int e = threadIdx.x; e < pairs; e += blockDim.x) {
        const int j = e / b.m, i = e - j * b.m;
        out[e] = dl_entry(g, b.t0 + i, b.s0 + j);
#pragma unroll
        for (int v = 1; v < 6; ++v) out[(size_t)v * pairs + e] = 0.0;
    }
}

// ---------------------------------------------------------------- geometry kernel
__global__ void geom_kernel(int M, const int32_t* __restrict__ perm, const int32_t* __restrict__ T,
                            const double* __restrict__ V, double* __restrict__ tri,
                            double* __restrict__ qp, double* __restrict__ qw)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    int t = perm[p];
    double v[9];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) v[3 * c + k] = V[3 * (size_t)T[3 * (size_t)t + c] + k];
#pragma unroll
    for (int c = 0; c < 9; ++c) tri[9 * (size_t)p + c] = v[c];
    double u[3], w[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        u[k] = v[3 + k] - v[k];
        w[k] = v[6 + k] - v[k];
    }
    double n0 = u[1] * w[2] - u[2] * w[1], n1 = u[2] * w[0] - u[0] * w[2], n2 = u[0] * w[1] - u[1] * w[0];
    double area = 0.5 * sqrt(n0 * n0 + n1 * n1 + n2 * n2);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
            qp[21 * (size_t)p + 3 * q + k] =
                c_lam[3 * q] * v[k] + c_lam[3 * q + 1] * v[3 + k] + c_lam[3 * q + 2] * v[6 + k];
        qw[7 * (size_t)p + q] = c_w7[q] * area * kInv4Pi;
    }
}

// ---------------------------------------------------------------- near field
// One CTA per near block; output per block [v][j][i] (i fastest), v = the six
// kernels V_11..V_33 (V_Delta is their trace).  qcount (optional) receives
// the quadrature work: [0] pairs on the whole-triangle 7-point rule, [1]
// subdivision leaves, [2] self pairs -- one atomic add per warp.
__global__ void __launch_bounds__(128) near_kernel(Geom g, const Blk* __restrict__ blks,
                                                   const int64_t* __restrict__ noff,
                                                   double* __restrict__ N,
                                                   unsigned long long* __restrict__ qcount)
{
    Blk b = blks[blockIdx.x];
    double* out = N + noff[blockIdx.x];
    int pairs = b.m * b.n;
    unsigned long long c_far = 0, c_leaf = 0, c_self = 0;
    for (int e = threadIdx.x; e < pairs; e += blockDim.x) {
        int j = e / b.m, i = e - j * b.m;
        double a[7];
        const int rule = entry7(g, b.t0 + i, b.s0 + j, a);
        c_far += rule == 0;
        c_self += rule < 0;
        c_leaf += rule > 0 ? (unsigned long long)rule : 0ull;
#pragma unroll
        for (int v = 0; v < 6; ++v) out[(size_t)v * pairs + e] = a[1 + v];
    }
    if (qcount) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c_far += __shfl_xor_sync(0xffffffffu, c_far, o);
            c_leaf += __shfl_xor_sync(0xffffffffu, c_leaf, o);
            c_self += __shfl_xor_sync(0xffffffffu, c_self, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(qcount, c_far);
            atomicAdd(qcount + 1, c_leaf);
            atomicAdd(qcount + 2, c_self);
        }
    }
}

// ---------------------------------------------------------------- batched ACA
struct AcaTask {
    int32_t blk, kern;
};

// device bytes of per-CTA ACA scratch per launch (the grid of a launch over
// very large blocks is reduced to stay within it)
constexpr size_t kAcaScratchBytes = size_t(4) << 30;

struct AcaParams {
    double fac;        // eps (1 - eta_stop) / (1 + eps)
    int32_t kmax;
    int32_t kcap_all;  // columns reserved per CTA in scratch
    int32_t mmax, nmax;
    // optional: entries evaluated, [0] V_Delta, [1] the V_kl (thread 0 of a
    // CTA adds its task's count once)
    unsigned long long* ecount = nullptr;
};

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_min_i(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

struct AcaShared {
    double su[kKmaxLimit];   // U[l][i_k] for the residual row
    double sv[kKmaxLimit];   // V[l][j_k] for the residual column
    double red[kAcaWarps][2 * kKmaxLimit + 2];
    double bc[4];
    int ibc[2];
    int task;
};

__device__ double block_max(AcaShared& sh, double v)
{
    v = warp_max(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh.red[w][0] = v;
    __syncthreads();
    double r = sh.red[0][0];
    for (int q = 1; q < kAcaWarps; ++q) r = fmax(r, sh.red[q][0]);
    return r;
}

__device__ void block_max2(AcaShared& sh, double& a, double& b)
{
    a = warp_max(a);
    b = warp_max(b);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) {
        sh.red[w][0] = a;
        sh.red[w][1] = b;
    }
    __syncthreads();
    double ra = sh.red[0][0], rb = sh.red[0][1];
    for (int q = 1; q < kAcaWarps; ++q) {
        ra = fmax(ra, sh.red[q][0]);
        rb = fmax(rb, sh.red[q][1]);
    }
    a = ra;
    b = rb;
}

__device__ int block_min_i(AcaShared& sh, int v)
{
    v = warp_min_i(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh.red[w][0] = (double)v;
    __syncthreads();
    double r = sh.red[0][0];
    for (int q = 1; q < kAcaWarps; ++q) r = fmin(r, sh.red[q][0]);
    return (int)r;
}

// next pivot row: the smallest row outside Z whose |u| is within the tie gap
// of the largest |u| outside Z; the smallest row outside Z if u vanishes there
__device__ int next_row(AcaShared& sh, const double* u, const unsigned char* Z, int m)
{
    double mx = 0.0;
    if (u)
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            if (!Z[i]) mx = fmax(mx, fabs(u[i]));
    mx = block_max(sh, mx);
    int cand = INT_MAX;
    if (mx > 0.0) {
        double thr = mx * (1.0 - kAcaTie);
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            if (!Z[i] && fabs(u[i]) >= thr) {
                cand = i;
                break;
            }
    } else {
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            if (!Z[i]) {
                cand = i;
                break;
            }
    }
    return block_min_i(sh, cand);
}

// Persistent batched ACA.  Each CTA takes tasks (admissible block, scalar
// kernel) from a global counter, largest blocks first, and runs Algorithm 1
// with its U / V columns in its own slice of `scratch`; the finished factors
// (U: m x k, then V: n x k, both column-major) are appended to `arena` at an
// offset taken with atomicAdd and repacked in block order afterwards.
// DL: the entries are the double layer's K_Delta (task kernel 0 only)
template <bool DL>
__global__ void __launch_bounds__(kAcaThreads) aca_kernel(
    Geom g, const AcaTask* __restrict__ tasks, int ntask, const Blk* __restrict__ blks,
    AcaParams prm, double* __restrict__ scratch, unsigned char* __restrict__ zscr,
    int* __restrict__ counter, double* __restrict__ arena, unsigned long long* __restrict__ arena_top,
    unsigned long long arena_cap, int32_t* __restrict__ out_rank, int64_t* __restrict__ out_off,
    int32_t* __restrict__ out_flags, AcaResume rs)
{
    __shared__ AcaShared sh;
    const int tid = threadIdx.x;
    const int B = blockDim.x;
    double* U = scratch + (size_t)blockIdx.x * (size_t)prm.kcap_all * (prm.mmax + prm.nmax);
    double* Vf = U + (size_t)prm.kcap_all * prm.mmax;
    unsigned char* Z = zscr + (size_t)blockIdx.x * prm.mmax;

    for (;;) {
        __syncthreads();
        if (tid == 0) sh.task = atomicAdd(counter, 1);
        __syncthreads();
        const int task = sh.task;
        if (task >= ntask) break;
        const AcaTask tk = tasks[task];
        const Blk b = blks[tk.blk];
        const int m = b.m, n = b.n, kern = tk.kern;
        const int ka = kern == 0 ? 0 : (kern <= 3 ? 0 : (kern <= 5 ? 1 : 2));
        const int kb = kern == 0 ? 0 : (kern <= 3 ? kern - 1 : (kern <= 5 ? kern - 3 : 2));
        int kcap = min(prm.kmax, min(m, n));
        int k = 0, nz = 0, flags = 0, irow = 0;
        double S2 = 0.0;
        const int64_t q7 = (int64_t)tk.blk * 7 + kern;
        const double* prevU = rs.k ? rs.prevU[q7] : nullptr;
        if (prevU) {
            // resume: the previous run's crosses, Z, next row and ||S||^2
            k = rs.k[q7];
            nz = rs.nz[q7];
            irow = rs.irow[q7];
            S2 = rs.S2[q7];
            const double* prevV = prevU + (size_t)k * m;
            for (int l = 0; l < k; ++l) {
                for (int i = tid; i < m; i += B) U[(size_t)l * m + i] = prevU[(size_t)l * m + i];
                for (int j = tid; j < n; j += B) Vf[(size_t)l * n + j] = prevV[(size_t)l * n + j];
            }
            for (int i = tid; i < m; i += B) Z[i] = rs.Z[rs.zoff[q7] + i];
        } else {
            for (int i = tid; i < m; i += B) Z[i] = 0;
        }
        __syncthreads();
        unsigned long long nent = 0;  // entries this task evaluates (thread 0)
        for (;;) {
            if (k >= prm.kmax) {
                flags |= 1;
                break;
            }
            nent += (unsigned long long)n;
            // residual row  v~ = A[i, s] - sum_{l<k} (u_l)_i v_l
            for (int l = tid; l < k; l += B) sh.su[l] = U[(size_t)l * m + irow];
            __syncthreads();
            double* vk = Vf + (size_t)k * n;
            double mraw = 0.0, mres = 0.0;
            for (int j = tid; j < n; j += B) {
                double a = DL ? dl_entry(g, b.t0 + irow, b.s0 + j) : entry1(g, b.t0 + irow, b.s0 + j, kern, ka, kb);
                double s = a;
                for (int l = 0; l < k; ++l) s -= sh.su[l] * Vf[(size_t)l * n + j];
                vk[j] = s;
                mraw = fmax(mraw, fabs(a));
                mres = fmax(mres, fabs(s));
            }
            block_max2(sh, mraw, mres);
            if (tid == 0) Z[irow] = 1;
            ++nz;
            if (!(mres > 0.0) || mres <= kAcaDelta * mraw) {
                // vanishing row: try another one
                if (nz == m) {
                    flags |= 2;
                    break;
                }
                __syncthreads();
                irow = next_row(sh, k > 0 ? U + (size_t)(k - 1) * m : nullptr, Z, m);
                if (irow >= m) {
                    flags |= 16;
                    break;
                }
                continue;
            }
            // pivot column: smallest j with |v~_j| >= (1 - tie) max
            double thr = mres * (1.0 - kAcaTie);
            int cand = INT_MAX;
            for (int j = tid; j < n; j += B)
                if (fabs(vk[j]) >= thr) {
                    cand = j;
                    break;
                }
            const int jk = block_min_i(sh, cand);
            if (jk >= n) {  // no finite pivot (non-finite entries): give up on this block
                flags |= 16;
                break;
            }
            const double inv = 1.0 / vk[jk];
            nent += (unsigned long long)m;
            __syncthreads();  // everyone has read the pivot before it is scaled
            double tvv = 0.0;
            for (int j = tid; j < n; j += B) {
                double s = vk[j] * inv;
                vk[j] = s;
                tvv += s * s;
            }
            for (int l = tid; l < k; l += B) sh.sv[l] = Vf[(size_t)l * n + jk];
            __syncthreads();
            // residual column  u_k = A[t, j_k] - sum_{l<k} (v_l)_{j_k} u_l
            double* uk = U + (size_t)k * m;
            double tuu = 0.0;
            for (int i = tid; i < m; i += B) {
                double a = DL ? dl_entry(g, b.t0 + i, b.s0 + jk) : entry1(g, b.t0 + i, b.s0 + jk, kern, ka, kb);
                double s = a;
                for (int l = 0; l < k; ++l) s -= sh.sv[l] * U[(size_t)l * m + i];
                uk[i] = s;
                tuu += s * s;
            }
            __syncthreads();
            // ||S_k||_F^2 = ||S_{k-1}||^2 + 2 sum_l (u_k.u_l)(v_l.v_k) + |u_k|^2 |v_k|^2
            const int w = tid >> 5, ln = tid & 31;
            for (int l = 0; l < k; ++l) {
                double pa = 0.0, pb = 0.0;
                for (int i = tid; i < m; i += B) pa += uk[i] * U[(size_t)l * m + i];
                for (int j = tid; j < n; j += B) pb += Vf[(size_t)l * n + j] * vk[j];
                pa = warp_sum(pa);
                pb = warp_sum(pb);
                if (ln == 0) {
                    sh.red[w][2 * l] = pa;
                    sh.red[w][2 * l + 1] = pb;
                }
            }
            tuu = warp_sum(tuu);
            tvv = warp_sum(tvv);
            if (ln == 0) {
                sh.red[w][2 * k] = tuu;
                sh.red[w][2 * k + 1] = tvv;
            }
            __syncthreads();
            if (tid < 32) {
                double cr = 0.0;
                for (int l = tid; l < k; l += 32) {
                    double a = 0.0, c = 0.0;
                    for (int q = 0; q < kAcaWarps; ++q) {
                        a += sh.red[q][2 * l];
                        c += sh.red[q][2 * l + 1];
                    }
                    cr += a * c;
                }
                cr = warp_sum(cr);
                if (tid == 0) {
                    double uu = 0.0, vv = 0.0;
                    for (int q = 0; q < kAcaWarps; ++q) {
                        uu += sh.red[q][2 * k];
                        vv += sh.red[q][2 * k + 1];
                    }
                    sh.bc[0] = cr;
                    sh.bc[1] = uu;
                    sh.bc[2] = vv;
                }
            }
            __syncthreads();
            const double uu = sh.bc[1], vv = sh.bc[2];
            S2 = S2 + 2.0 * sh.bc[0] + uu * vv;
            ++k;
            if (sqrt(uu * vv) <= prm.fac * sqrt(fmax(S2, 0.0))) break;
            if (nz == m) {
                flags |= 2;
                break;
            }
            // at kmax below min(|t|, |s|) a resumable run (ACA on demand) also
            // finds the next row, so that a later run can go on from it; it
            // then stops at the top of the loop (flag 1)
            if (k >= kcap && !(rs.k && kcap == prm.kmax && prm.kmax < min(m, n))) {
                flags |= 4;
                break;
            }
            __syncthreads();
            irow = next_row(sh, uk, Z, m);
            if (irow >= m) {
                flags |= 16;
                break;
            }
        }
        // append the factors to the arena
        __syncthreads();
        if (rs.k) {
            // the state a later run resumes from
            if (tid == 0) {
                rs.k[q7] = k;
                rs.nz[q7] = nz;
                rs.irow[q7] = irow;
                rs.flags[q7] = flags;
                rs.S2[q7] = S2;
            }
            for (int i = tid; i < m; i += B) rs.Z[rs.zoff[q7] + i] = Z[i];
        }
        if (tid == 0) {
            unsigned long long need = (unsigned long long)k * (m + n);
            unsigned long long off = atomicAdd(arena_top, need);
            if (off + need > arena_cap) {
                sh.ibc[0] = -1;
            } else {
                sh.ibc[0] = 0;
                out_off[task] = (int64_t)off;
            }
            out_rank[task] = k;
        }
        __syncthreads();
        if (sh.ibc[0] < 0) {
            flags |= 8;
        } else if (k > 0) {
            double* dst = arena + out_off[task];
            for (int l = 0; l < k; ++l) {
                for (int i = tid; i < m; i += B) dst[(size_t)l * m + i] = U[(size_t)l * m + i];
            }
            double* dv = dst + (size_t)k * m;
            for (int l = 0; l < k; ++l) {
                for (int j = tid; j < n; j += B) dv[(size_t)l * n + j] = Vf[(size_t)l * n + j];
            }
        }
        if (tid == 0) {
            out_flags[task] = flags;
            if (prm.ecount) atomicAdd(prm.ecount + (kern == 0 ? 0 : 1), nent);
        }
    }
}

// copy finished factors from the arena into the block-ordered U / V arenas
__global__ void repack_kernel(const AcaTask* __restrict__ tasks, int ntask,
                              const Blk* __restrict__ blks, const int32_t* __restrict__ rank,
                              const int64_t* __restrict__ off, const double* __restrict__ arena,
                              int64_t cap, const double* __restrict__ arena2,
                              const int64_t* __restrict__ uoff, const int64_t* __restrict__ voff,
                              double* __restrict__ U, double* __restrict__ V)
{
    int task = blockIdx.x;
    if (task >= ntask) return;
    AcaTask tk = tasks[task];
    int k = rank[task];
    if (k == 0) return;
    Blk b = blks[tk.blk];
    const int64_t o = off[task];
    const double* src = o < cap ? arena + o : arena2 + (o - cap);
    size_t q = (size_t)tk.blk * 7 + tk.kern;
    double* du = U + uoff[q];
    double* dv = V + voff[q];
    size_t nu = (size_t)k * b.m, nv = (size_t)k * b.n;
    for (size_t e = threadIdx.x; e < nu; e += blockDim.x) du[e] = src[e];
    for (size_t e = threadIdx.x; e < nv; e += blockDim.x) dv[e] = src[nu + e];
}

// allocate max(bytes, 16) and copy exactly `bytes` (an empty list is a valid,
// never-read device buffer)
int upload(hm_matrix& H, DevBuf& d, const void* src, size_t bytes)
{
    d.bytes = std::max<size_t>(bytes, 16);
    d.p = H.alloc.alloc(d.bytes);
    if (!d.p) return fail(HM_ENOMEM, "device allocation of %zu bytes failed", d.bytes);
    if (bytes) HM_CUDA(cudaMemcpyAsync(d.p, src, bytes, cudaMemcpyHostToDevice, H.alloc.stream));
    return HM_OK;
}

int dalloc(hm_matrix& H, DevBuf& d, size_t bytes)
{
    d.bytes = bytes;
    d.p = H.alloc.alloc(bytes);
    if (!d.p) return fail(HM_ENOMEM, "device allocation of %zu bytes failed", bytes);
    return HM_OK;
}

struct TmpBuf {
    hm_matrix& H;
    DevBuf b;
    explicit TmpBuf(hm_matrix& h) : H(h) {}
    ~TmpBuf() { H.alloc.release(b.p, b.bytes); }
};

}  // namespace

// ------------------------------------------------------------------------
int aca_on_demand(hm_matrix& H, const std::vector<int32_t>& bk, int kmax, cudaStream_t s, DevBuf& out,
                  std::vector<int32_t>& rank, std::vector<int64_t>& off, const AcaResume* resume,
                  std::vector<int32_t>* flags_out, size_t cap_hint)
{
    const int64_t nt = (int64_t)bk.size();
    rank.assign((size_t)nt, 0);
    off.assign((size_t)nt, 0);
    if (flags_out) flags_out->assign((size_t)nt, 0);
    if (nt == 0) return HM_OK;
    if (!H.g_coll.p) return fail(HM_EINVAL, "ACA on demand: the matrix keeps no geometry");
    if (kmax < 1) return fail(HM_EINVAL, "ACA on demand: kmax %d < 1", kmax);
    Geom g{H.g_coll.as<double>(), H.g_tri.as<double>(), H.g_qp.as<double>(), H.g_qw.as<double>(),
           H.g_diam.as<double>(), H.rect ? H.g_rows.as<double>() : H.g_coll.as<double>(), H.rect ? 0 : 1};
    if (H.dl) {
        g.nrm = H.g_nrm.as<double>();
        g.star_ptr = H.d_star_ptr.as<int32_t>();
        g.star = H.d_star.as<int32_t>();
    }
    auto aca = H.dl ? aca_kernel<true> : aca_kernel<false>;
    // tasks by decreasing |t| + |s| (as at assembly); ord maps back
    std::vector<int64_t> ord((size_t)nt);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) {
        const Blk& a = H.adm_h[(size_t)(bk[(size_t)x] / 7)];
        const Blk& c = H.adm_h[(size_t)(bk[(size_t)y] / 7)];
        return (int64_t)a.m + a.n > (int64_t)c.m + c.n;
    });
    std::vector<AcaTask> tasks((size_t)nt);
    unsigned long long cap = 1;  // every task's factors fit: kmax (m + n) each at most
    for (int64_t q = 0; q < nt; ++q) {
        const int32_t v = bk[(size_t)ord[(size_t)q]];
        tasks[(size_t)q] = AcaTask{v / 7, v % 7};
        const Blk& b = H.adm_h[(size_t)(v / 7)];
        cap += (unsigned long long)std::min(kmax, std::min(b.m, b.n)) * (unsigned long long)(b.m + b.n);
    }
    const double eps = H.prm.aca_eps;
    const double fac = eps * (1.0 - H.prm.aca_eta_stop) / (1.0 + eps);
    int dev = 0, nsm = 0, occ = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, aca, kAcaThreads, 0));
    const int64_t full_grid = (int64_t)nsm * std::max(1, std::min(occ, 4));
    struct Cls {
        int64_t i0, i1, grid;
        AcaParams prm;
    };
    std::vector<Cls> cls;
    size_t scr_bytes = 0, z_bytes = 0;
    for (int64_t i0 = 0; i0 < nt;) {
        const Blk& b0 = H.adm_h[(size_t)tasks[(size_t)i0].blk];
        const int64_t half = ((int64_t)b0.m + b0.n) / 2;
        int64_t i1 = i0 + 1;
        while (i1 < nt) {
            const Blk& b = H.adm_h[(size_t)tasks[(size_t)i1].blk];
            if ((int64_t)b.m + b.n <= half) break;
            ++i1;
        }
        Cls c;
        c.i0 = i0;
        c.i1 = i1;
        int mmax = 1, nmax = 1, kc = 1;
        for (int64_t q = i0; q < i1; ++q) {
            const Blk& b = H.adm_h[(size_t)tasks[(size_t)q].blk];
            mmax = std::max(mmax, b.m);
            nmax = std::max(nmax, b.n);
            kc = std::max(kc, std::min(b.m, b.n));
        }
        c.prm.fac = fac;
        c.prm.kmax = kmax;
        c.prm.kcap_all = std::max(1, std::min(kc, kmax));
        c.prm.mmax = mmax;
        c.prm.nmax = nmax;
        const size_t per_cta = (size_t)c.prm.kcap_all * (size_t)(mmax + nmax) * 8;
        c.grid = std::max<int64_t>(1, std::min<int64_t>({full_grid, i1 - i0, (int64_t)(kAcaScratchBytes / per_cta)}));
        scr_bytes = std::max(scr_bytes, (size_t)c.grid * per_cta);
        z_bytes = std::max(z_bytes, (size_t)c.grid * (size_t)mmax);
        cls.push_back(c);
        i0 = i1;
    }
    int rc;
    TmpBuf dscr(H), dz(H), dtask(H), dcnt(H), dtop(H), drank(H), doff(H), dflag(H);
    if ((rc = dalloc(H, dscr.b, scr_bytes))) return rc;
    if ((rc = dalloc(H, dz.b, z_bytes))) return rc;
    if ((rc = upload(H, dtask.b, tasks.data(), tasks.size() * sizeof(AcaTask)))) return rc;
    if ((rc = dalloc(H, dcnt.b, 64))) return rc;
    if ((rc = dalloc(H, dtop.b, 64))) return rc;
    if ((rc = dalloc(H, drank.b, (size_t)nt * 4))) return rc;
    if ((rc = dalloc(H, doff.b, (size_t)nt * 8))) return rc;
    if ((rc = dalloc(H, dflag.b, (size_t)nt * 4))) return rc;
    std::vector<int32_t> r((size_t)nt), f((size_t)nt);
    std::vector<int64_t> o((size_t)nt);
    auto run_all = [&](unsigned long long arena_cap) -> int {
        int rc2;
        if ((rc2 = dalloc(H, out, (size_t)arena_cap * 8))) return rc2;
        HM_CUDA(cudaMemsetAsync(dtop.b.p, 0, 64, s));
        for (const Cls& c : cls) {
            HM_CUDA(cudaMemsetAsync(dcnt.b.p, 0, 64, s));
            aca<<<(unsigned)c.grid, kAcaThreads, 0, s>>>(
                g, dtask.b.as<AcaTask>() + c.i0, (int)(c.i1 - c.i0), H.d_adm.as<Blk>(), c.prm, dscr.b.as<double>(),
                dz.b.as<unsigned char>(), dcnt.b.as<int>(), out.as<double>(), dtop.b.as<unsigned long long>(),
                arena_cap, drank.b.as<int32_t>() + c.i0, doff.b.as<int64_t>() + c.i0, dflag.b.as<int32_t>() + c.i0,
                resume ? *resume : AcaResume{});
            HM_CUDA(cudaGetLastError());
        }
        HM_CUDA(cudaMemcpyAsync(r.data(), drank.b.p, (size_t)nt * 4, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaMemcpyAsync(o.data(), doff.b.p, (size_t)nt * 8, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaMemcpyAsync(f.data(), dflag.b.p, (size_t)nt * 4, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        return HM_OK;
    };
    // with a hint below the bound, tasks that do not fit are detected (flag 8)
    // and the whole batch runs again into an arena of the exact size (the
    // ranks are known by then; a resumable run is never hinted, so running it
    // twice is safe: ACA is deterministic)
    const bool hinted = cap_hint > 0 && cap_hint < cap && !resume;
    if ((rc = run_all(hinted ? (unsigned long long)cap_hint : cap))) return rc;
    if (hinted) {
        unsigned long long need = 1;
        bool over = false;
        for (int64_t q = 0; q < nt; ++q) {
            const Blk& b = H.adm_h[(size_t)tasks[(size_t)q].blk];
            need += (unsigned long long)r[(size_t)q] * (unsigned long long)(b.m + b.n);
            over = over || (f[(size_t)q] & 8);
        }
        if (over) {
            H.alloc.release(out.p, out.bytes);
            out = DevBuf{};
            if ((rc = run_all(need))) return rc;
        }
    }
    for (int64_t q = 0; q < nt; ++q) {
        if (f[(size_t)q] & 8) return fail(HM_EDEVICE, "ACA on demand: arena overflow");
        rank[(size_t)ord[(size_t)q]] = r[(size_t)q];
        off[(size_t)ord[(size_t)q]] = o[(size_t)q];
        if (flags_out) (*flags_out)[(size_t)ord[(size_t)q]] = f[(size_t)q];
    }
    return HM_OK;
}

// ------------------------------------------------------------------------
std::vector<FwdTcUnit> tc_units(const std::vector<FwdUnit>& units, const std::vector<FwdGroup>& groups)
{
    std::vector<FwdTcUnit> out(units.size());
    for (size_t i = 0; i < units.size(); ++i) {
        const FwdUnit& u = units[i];
        const FwdGroup& g = groups[(size_t)u.group];
        FwdTcUnit t{};
        // the unit's tiles are contiguous: after the full row chunks above it
        // and the units to its left in its row chunk (16-bit layout of V)
        t.v0 = g.vbase + (int64_t)u.j0 * g.Cs + (int64_t)((u.nrows + 15) & ~15) * u.c0;
        t.z0 = u.zcol0 >= 0 ? u.zcol0 + (int64_t)u.chunk * g.Cs + u.c0 : -1;
        t.x0 = g.s0 + u.j0;
        t.d0 = g.dbase + u.c0;
        t.ld8 = u.ncols * 8;
        t.nrows = (int16_t)u.nrows;
        t.ncols = (int16_t)u.ncols;
        t.mesh = g.mesh;
        out[i] = t;
    }
    return out;
}

static int upload_tables(cudaStream_t s)
{
    double lam[21], w7[7], gx[kGL], gw[kGL];
    radon_table(lam, w7);
    gauss_legendre_table(kGL, gx, gw);
    HM_CUDA(cudaMemcpyToSymbolAsync(c_lam, lam, sizeof lam, 0, cudaMemcpyHostToDevice, s));
    HM_CUDA(cudaMemcpyToSymbolAsync(c_w7, w7, sizeof w7, 0, cudaMemcpyHostToDevice, s));
    HM_CUDA(cudaMemcpyToSymbolAsync(c_glx, gx, sizeof gx, 0, cudaMemcpyHostToDevice, s));
    HM_CUDA(cudaMemcpyToSymbolAsync(c_glw, gw, sizeof gw, 0, cudaMemcpyHostToDevice, s));
    return HM_OK;
}

// the triangles' geometry in cluster order, kept with the matrix: column
// permutation, centroids, squared diameters, vertices and 7-point rules
static int upload_geometry(const hm_tree& tr, hm_matrix& H)
{
    cudaStream_t s = H.alloc.stream;
    const int64_t M = tr.M;
    std::vector<int32_t> perm32((size_t)M);
    std::vector<double> coll((size_t)(3 * M)), diam2((size_t)M);
    for (int64_t p = 0; p < M; ++p) {
        int64_t t = tr.perm[(size_t)p];
        perm32[(size_t)p] = (int32_t)t;
        for (int k = 0; k < 3; ++k) coll[(size_t)(3 * p + k)] = tr.coll[(size_t)(3 * t + k)];
        const double* v[3];
        for (int c = 0; c < 3; ++c) v[c] = &tr.V[3 * (size_t)tr.T[(size_t)(3 * t + c)]];
        double dm = 0.0;
        for (int e = 0; e < 3; ++e) {
            const double* a = v[e];
            const double* b = v[(e + 1) % 3];
            double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
            double q = d0 * d0 + d1 * d1 + d2 * d2;  // host code: no contraction
            dm = std::max(dm, q);
        }
        diam2[(size_t)p] = dm;
    }
    int rc;
    if ((rc = upload(H, H.d_perm, perm32.data(), perm32.size() * 4))) return rc;
    // the geometry of the entries stays with the matrix (ACA on demand)
    TmpBuf dV(H), dT(H);
    if ((rc = upload(H, dV.b, tr.V.data(), tr.V.size() * 8))) return rc;
    if ((rc = upload(H, dT.b, tr.T.data(), tr.T.size() * 4))) return rc;
    if ((rc = upload(H, H.g_coll, coll.data(), coll.size() * 8))) return rc;
    if ((rc = upload(H, H.g_diam, diam2.data(), diam2.size() * 8))) return rc;
    if ((rc = dalloc(H, H.g_tri, (size_t)M * 9 * 8))) return rc;
    if ((rc = dalloc(H, H.g_qp, (size_t)M * 21 * 8))) return rc;
    if ((rc = dalloc(H, H.g_qw, (size_t)M * 7 * 8))) return rc;
    geom_kernel<<<(unsigned)((M + 127) / 128), 128, 0, s>>>((int)M, H.d_perm.as<int32_t>(),
                                                            dT.b.as<int32_t>(), dV.b.as<double>(),
                                                            H.g_tri.as<double>(), H.g_qp.as<double>(),
                                                            H.g_qw.as<double>());
    HM_CUDA(cudaGetLastError());
    return HM_OK;
}

int assemble_points_device(const hm_tree& tr, hm_matrix& H);
// FNV-1a over the mesh's vertex coordinates and triangles: matrices built on
// the same mesh (the double layer's two operators) carry the same value
static uint64_t mesh_fingerprint(const hm_tree& tr)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    };
    mix(tr.V.data(), tr.V.size() * sizeof(double));
    mix(tr.T.data(), tr.T.size() * sizeof(int32_t));
    return h;
}

// The double layer's columns (Section 4.2, Eq. (Kh)): the vertex tree `tr`
// over the triangles of tr.src.  Rows are the triangles' collocation points
// (cluster order of tr.src, whose geometry upload_geometry has placed);
// columns the vertices in tr's cluster order.  Per triangle its unit normal
// and twice its area (the cross product (p1 - p0) x (p2 - p0) in the
// triangle's own vertex order), per vertex its star sorted by triangle id,
// and the triangles' vertex ids for the surface curls.
static int upload_dl_geometry(const hm_tree& tr, hm_matrix& H)
{
    const hm_tree& src = *tr.src;
    const int64_t M = src.M, nv = tr.M;
    int rc;
    // rows: the triangle perm (upload_geometry put it in d_perm) and the
    // centroids in cluster order
    std::vector<int32_t> rperm((size_t)M), vperm((size_t)nv), tpos((size_t)M);
    std::vector<double> rows((size_t)(3 * M)), nrm((size_t)(4 * M));
    for (int64_t p = 0; p < M; ++p) {
        const int64_t t = src.perm[(size_t)p];
        rperm[(size_t)p] = (int32_t)t;
        tpos[(size_t)t] = (int32_t)p;
        for (int k = 0; k < 3; ++k) rows[(size_t)(3 * p + k)] = src.coll[(size_t)(3 * t + k)];
        const double* p0 = &src.V[3 * (size_t)src.T[(size_t)(3 * t)]];
        const double* p1 = &src.V[3 * (size_t)src.T[(size_t)(3 * t + 1)]];
        const double* p2 = &src.V[3 * (size_t)src.T[(size_t)(3 * t + 2)]];
        const double e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
        const double e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
        const double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                             e1[0] * e2[1] - e1[1] * e2[0]};
        const double len = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        if (!(len > 0.0)) return fail(HM_EINVAL, "double layer: triangle %lld is degenerate", (long long)t);
        for (int k = 0; k < 3; ++k) nrm[(size_t)(4 * p + k)] = c[k] / len;
        nrm[(size_t)(4 * p + 3)] = len;
    }
    // stars: for the vertex at cluster position q, (triangle position, corner)
    // of every triangle holding it, by increasing triangle id
    std::vector<int32_t> vpos((size_t)nv), cnt((size_t)nv + 1, 0);
    for (int64_t q = 0; q < nv; ++q) {
        vperm[(size_t)q] = (int32_t)tr.perm[(size_t)q];
        vpos[(size_t)tr.perm[(size_t)q]] = (int32_t)q;
    }
    for (int64_t t = 0; t < M; ++t)
        for (int c = 0; c < 3; ++c) ++cnt[(size_t)vpos[(size_t)src.T[(size_t)(3 * t + c)]] + 1];
    for (int64_t q = 0; q < nv; ++q) cnt[(size_t)q + 1] += cnt[(size_t)q];
    std::vector<int32_t> star((size_t)cnt[(size_t)nv]), fill(cnt.begin(), cnt.end() - 1);
    for (int64_t t = 0; t < M; ++t)
        for (int c = 0; c < 3; ++c) {
            const int32_t q = vpos[(size_t)src.T[(size_t)(3 * t + c)]];
            star[(size_t)fill[(size_t)q]++] = tpos[(size_t)t] * 4 + c;
        }
    if ((rc = upload(H, H.d_rperm, rperm.data(), rperm.size() * 4))) return rc;
    H.alloc.release(H.d_perm.p, H.d_perm.bytes);
    H.d_perm = DevBuf{};
    if ((rc = upload(H, H.d_perm, vperm.data(), vperm.size() * 4))) return rc;
    if ((rc = upload(H, H.g_rows, rows.data(), rows.size() * 8))) return rc;
    if ((rc = upload(H, H.g_nrm, nrm.data(), nrm.size() * 8))) return rc;
    if ((rc = upload(H, H.d_star_ptr, cnt.data(), cnt.size() * 4))) return rc;
    if ((rc = upload(H, H.d_star, star.data(), star.size() * 4))) return rc;
    if ((rc = upload(H, H.d_tris, src.T.data(), src.T.size() * 4))) return rc;
    if ((rc = dalloc(H, H.dl_w, (size_t)(3 * M) * 8))) return rc;
    return HM_OK;
}


int assemble_device(const hm_tree& tr, hm_matrix& H)
{
    if (tr.kind == 1 || tr.kind == 2) return assemble_points_device(tr, H);
    cudaStream_t s = H.alloc.stream;
    const int64_t M = tr.M;
    H.M = M;
    H.Mr = M;
    int rc;
    if ((rc = upload_tables(s))) return rc;
    if ((rc = upload_geometry(tr, H))) return rc;
    H.mesh_fp = mesh_fingerprint(tr);
    Geom g{H.g_coll.as<double>(), H.g_tri.as<double>(), H.g_qp.as<double>(), H.g_qw.as<double>(),
           H.g_diam.as<double>(), H.g_coll.as<double>(), 1};

    // ---- block lists
    auto blk_of = [&](const std::array<int64_t, 2>& ts) {
        const Node& a = tr.nodes[(size_t)ts[0]];
        const Node& c = tr.nodes[(size_t)ts[1]];
        return Blk{(int32_t)a.lo, (int32_t)(a.hi - a.lo), (int32_t)c.lo, (int32_t)(c.hi - c.lo)};
    };
    H.nadm = (int64_t)tr.adm.size();
    H.nnear = (int64_t)tr.near_blocks.size();
    H.adm_h.resize((size_t)H.nadm);
    H.near_h.resize((size_t)H.nnear);
    for (int64_t b = 0; b < H.nadm; ++b) H.adm_h[(size_t)b] = blk_of(tr.adm[(size_t)b]);
    for (int64_t b = 0; b < H.nnear; ++b) H.near_h[(size_t)b] = blk_of(tr.near_blocks[(size_t)b]);
    if ((rc = upload(H, H.d_adm, H.adm_h.data(), H.adm_h.size() * sizeof(Blk)))) return rc;
    if ((rc = upload(H, H.d_near, H.near_h.data(), H.near_h.size() * sizeof(Blk)))) return rc;

    cudaEvent_t ev[4];
    for (auto& e : ev) HM_CUDA(cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard()
        {
            for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]);
        }
    } evg{ev};

    // ---- near field
    H.noff_h.resize((size_t)H.nnear);
    int64_t ntot = 0;
    for (int64_t b = 0; b < H.nnear; ++b) {
        H.noff_h[(size_t)b] = ntot;
        ntot += 6 * (int64_t)H.near_h[(size_t)b].m * H.near_h[(size_t)b].n;
    }
    H.n_total = ntot;
    if ((rc = upload(H, H.d_noff, H.noff_h.data(), H.noff_h.size() * 8))) return rc;
    if ((rc = dalloc(H, H.N64, (size_t)std::max<int64_t>(ntot, 1) * 8))) return rc;
    // assembly work counters: near-field rules [0..2], ACA entries [3..4]
    TmpBuf dqc(H);
    if ((rc = dalloc(H, dqc.b, 64))) return rc;
    HM_CUDA(cudaMemsetAsync(dqc.b.p, 0, 64, s));
    unsigned long long* qc = dqc.b.as<unsigned long long>();
    HM_CUDA(cudaEventRecord(ev[0], s));
    if (H.nnear > 0) {
        near_kernel<<<(unsigned)H.nnear, 128, 0, s>>>(g, H.d_near.as<Blk>(), H.d_noff.as<int64_t>(),
                                                      H.N64.as<double>(), qc);
        HM_CUDA(cudaGetLastError());
    }
    HM_CUDA(cudaEventRecord(ev[1], s));

    // ---- batched ACA
    H.rank_h.assign((size_t)H.nadm * 7, 0);
    H.flags_h.assign((size_t)H.nadm * 7, 0);
    // A scalar kernel with factor (x - y)_a vanishes identically on a block
    // whose clusters' vertices all share coordinate a: exact rank 0 (what
    // Algorithm 1 reaches in exact arithmetic once Z = t), no ACA task.
    static const int kp[7] = {-1, 0, 0, 0, 1, 1, 2}, kq[7] = {-1, 0, 1, 2, 1, 2, 2};
    std::vector<AcaTask> tasks;
    tasks.reserve((size_t)H.nadm * 7);
    for (int64_t b = 0; b < H.nadm; ++b) {
        const Node& nt = tr.nodes[(size_t)tr.adm[(size_t)b][0]];
        const Node& ns = tr.nodes[(size_t)tr.adm[(size_t)b][1]];
        for (int k = 0; k < 7; ++k) {
            bool zero = false;
            if (k > 0)
                for (int a : {kp[k], kq[k]})
                    if (nt.bmin[a] == nt.bmax[a] && ns.bmin[a] == ns.bmax[a] && nt.bmin[a] == ns.bmin[a])
                        zero = true;
            if (zero)
                H.flags_h[(size_t)(b * 7 + k)] = 32;
            else
                tasks.push_back(AcaTask{(int32_t)b, k});
        }
    }
    if (H.prm.flags & HM_DEFER_ACA) {
        // the adaptive product runs Algorithm 1 on demand (hm_amvm)
        tasks.clear();
        H.aca_deferred = true;
    }
    const int64_t ntask = (int64_t)tasks.size();
    std::stable_sort(tasks.begin(), tasks.end(), [&](const AcaTask& x, const AcaTask& y) {
        const Blk& a = H.adm_h[(size_t)x.blk];
        const Blk& c = H.adm_h[(size_t)y.blk];
        return (int64_t)a.m + a.n > (int64_t)c.m + c.n;
    });
    std::vector<int32_t> trank((size_t)ntask, 0), tflags((size_t)ntask, 0);
    std::vector<int64_t> toff((size_t)ntask, 0);
    TmpBuf darena(H), darena2(H), dscr(H), dz(H), dtask(H), dcnt(H), dtop(H), drank(H), doff(H), dflag(H);
    unsigned long long cap = 0;  // elements of darena; offsets >= cap lie in darena2
    if (ntask > 0) {
        double est = 0.0;
        // first guess of the factor arena: rank 12 per block and kernel (the
        // measured means are 6-9 at eps 1e-4), at most 60% of the free
        // device memory; tasks that do not fit are re-run into an arena of
        // the exact size below
        for (const Blk& b : H.adm_h) est += 7.0 * (b.m + b.n) * std::min(12, std::min(b.m, b.n));
        {
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) est = std::min(est, 0.6 * (double)fr / 8.0 / 1.1);
            else cudaGetLastError();
        }
        const double eps = H.prm.aca_eps;
        const double fac = eps * (1.0 - H.prm.aca_eta_stop) / (1.0 + eps);
        int dev = 0, nsm = 0, occ = 0;
        HM_CUDA(cudaGetDevice(&dev));
        HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        HM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, aca_kernel<false>, kAcaThreads, 0));
        const int64_t full_grid = (int64_t)nsm * std::max(1, std::min(occ, 4));
        // Launch classes over the tasks (sorted by decreasing |t| + |s|): a
        // class ends where blocks are half the size of its first one.  Each
        // CTA's scratch holds the largest block of its class, and a class's
        // grid is bounded so that all its scratch fits kAcaScratchBytes.
        struct AcaClass {
            int64_t i0, i1, grid;
            AcaParams prm;
        };
        std::vector<AcaClass> classes;
        size_t scr_bytes = 0, z_bytes = 0;
        auto make_class = [&](const std::vector<AcaTask>& tl, int64_t i0, int64_t i1) {
            AcaClass c;
            c.i0 = i0;
            c.i1 = i1;
            int mmax = 1, nmax = 1, kc = 1;
            for (int64_t q = i0; q < i1; ++q) {
                const Blk& b = H.adm_h[(size_t)tl[(size_t)q].blk];
                mmax = std::max(mmax, b.m);
                nmax = std::max(nmax, b.n);
                kc = std::max(kc, std::min(b.m, b.n));
            }
            c.prm.fac = fac;
            c.prm.kmax = H.prm.kmax;
            c.prm.kcap_all = std::max(1, std::min(kc, H.prm.kmax));
            c.prm.mmax = mmax;
            c.prm.nmax = nmax;
            const size_t per_cta = (size_t)c.prm.kcap_all * (size_t)(mmax + nmax) * 8;
            c.grid = std::max<int64_t>(1, std::min<int64_t>({full_grid, i1 - i0, (int64_t)(kAcaScratchBytes / per_cta)}));
            scr_bytes = std::max(scr_bytes, (size_t)c.grid * per_cta);
            z_bytes = std::max(z_bytes, (size_t)c.grid * (size_t)mmax);
            return c;
        };
        auto split = [&](const std::vector<AcaTask>& tl, std::vector<AcaClass>& out) {
            int64_t i0 = 0;
            const int64_t nt = (int64_t)tl.size();
            while (i0 < nt) {
                const Blk& b0 = H.adm_h[(size_t)tl[(size_t)i0].blk];
                const int64_t half = ((int64_t)b0.m + b0.n) / 2;
                int64_t i1 = i0 + 1;
                while (i1 < nt) {
                    const Blk& b = H.adm_h[(size_t)tl[(size_t)i1].blk];
                    if ((int64_t)b.m + b.n <= half) break;
                    ++i1;
                }
                out.push_back(make_class(tl, i0, i1));
                i0 = i1;
            }
        };
        split(tasks, classes);
        if ((rc = dalloc(H, dscr.b, scr_bytes))) return rc;
        if ((rc = dalloc(H, dz.b, z_bytes))) return rc;
        if ((rc = upload(H, dtask.b, tasks.data(), tasks.size() * sizeof(AcaTask)))) return rc;
        if ((rc = dalloc(H, dcnt.b, 64))) return rc;
        if ((rc = dalloc(H, dtop.b, 64))) return rc;
        if ((rc = dalloc(H, drank.b, (size_t)ntask * 4))) return rc;
        if ((rc = dalloc(H, doff.b, (size_t)ntask * 8))) return rc;
        if ((rc = dalloc(H, dflag.b, (size_t)ntask * 4))) return rc;
        cap = (unsigned long long)(est * 1.1) + (1ull << 20);
        if ((rc = dalloc(H, darena.b, (size_t)cap * 8))) return rc;
        HM_CUDA(cudaMemsetAsync(dtop.b.p, 0, 64, s));
        for (const AcaClass& c : classes) {
            HM_CUDA(cudaMemsetAsync(dcnt.b.p, 0, 64, s));
            AcaParams cp = c.prm;
            cp.ecount = qc + 3;  // the first run of every task (not a re-run into the exact arena)
            aca_kernel<false><<<(unsigned)c.grid, kAcaThreads, 0, s>>>(
                g, dtask.b.as<AcaTask>() + c.i0, (int)(c.i1 - c.i0), H.d_adm.as<Blk>(), cp,
                dscr.b.as<double>(), dz.b.as<unsigned char>(), dcnt.b.as<int>(), darena.b.as<double>(),
                dtop.b.as<unsigned long long>(), cap, drank.b.as<int32_t>() + c.i0, doff.b.as<int64_t>() + c.i0,
                dflag.b.as<int32_t>() + c.i0, AcaResume{});
            HM_CUDA(cudaGetLastError());
        }
        HM_CUDA(cudaMemcpyAsync(trank.data(), drank.b.p, (size_t)ntask * 4, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaMemcpyAsync(toff.data(), doff.b.p, (size_t)ntask * 8, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaMemcpyAsync(tflags.data(), dflag.b.p, (size_t)ntask * 4, cudaMemcpyDeviceToHost, s));
        HM_CUDA(cudaStreamSynchronize(s));
        // tasks whose factors did not fit: run them again into a second arena
        // of the exact size (ACA is deterministic, so the result is the same)
        std::vector<AcaTask> redo;
        std::vector<int64_t> redo_idx;
        unsigned long long need = 0;
        for (int64_t q = 0; q < ntask; ++q)
            if (tflags[(size_t)q] & 8) {
                redo.push_back(tasks[(size_t)q]);
                redo_idx.push_back(q);
                const Blk& b = H.adm_h[(size_t)tasks[(size_t)q].blk];
                need += (unsigned long long)trank[(size_t)q] * (b.m + b.n);
            }
        if (!redo.empty()) {
            TmpBuf t2(H), r2(H), o2(H), f2(H);
            DevBuf& a2 = darena2.b;
            if ((rc = dalloc(H, a2, (size_t)(need + 1) * 8))) return rc;
            if ((rc = upload(H, t2.b, redo.data(), redo.size() * sizeof(AcaTask)))) return rc;
            if ((rc = dalloc(H, r2.b, redo.size() * 4))) return rc;
            if ((rc = dalloc(H, o2.b, redo.size() * 8))) return rc;
            if ((rc = dalloc(H, f2.b, redo.size() * 4))) return rc;
            HM_CUDA(cudaMemsetAsync(dtop.b.p, 0, 64, s));
            // the re-run tasks keep their decreasing size order; classes as above,
            // each grid bounded by the scratch already allocated
            std::vector<AcaClass> rcl;
            split(redo, rcl);
            for (AcaClass& c : rcl) {
                const size_t per_cta = (size_t)c.prm.kcap_all * (size_t)(c.prm.mmax + c.prm.nmax) * 8;
                c.grid = std::max<int64_t>(1, std::min<int64_t>({c.grid, (int64_t)(dscr.b.bytes / per_cta),
                                                                 (int64_t)(dz.b.bytes / (size_t)c.prm.mmax)}));
                HM_CUDA(cudaMemsetAsync(dcnt.b.p, 0, 64, s));
                aca_kernel<false><<<(unsigned)c.grid, kAcaThreads, 0, s>>>(
                    g, t2.b.as<AcaTask>() + c.i0, (int)(c.i1 - c.i0), H.d_adm.as<Blk>(), c.prm, dscr.b.as<double>(),
                    dz.b.as<unsigned char>(), dcnt.b.as<int>(), a2.as<double>(), dtop.b.as<unsigned long long>(),
                    need + 1, r2.b.as<int32_t>() + c.i0, o2.b.as<int64_t>() + c.i0, f2.b.as<int32_t>() + c.i0,
                    AcaResume{});
                HM_CUDA(cudaGetLastError());
            }
            // the re-run results: offsets past `cap` address the second arena
            std::vector<int32_t> rr(redo.size()), ff(redo.size());
            std::vector<int64_t> oo(redo.size());
            HM_CUDA(cudaMemcpyAsync(rr.data(), r2.b.p, rr.size() * 4, cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaMemcpyAsync(oo.data(), o2.b.p, oo.size() * 8, cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaMemcpyAsync(ff.data(), f2.b.p, ff.size() * 4, cudaMemcpyDeviceToHost, s));
            HM_CUDA(cudaStreamSynchronize(s));
            for (size_t q = 0; q < redo.size(); ++q) {
                size_t t = (size_t)redo_idx[q];
                trank[t] = rr[q];
                toff[t] = (int64_t)cap + oo[q];
                tflags[t] = ff[q];
            }
            if ((rc = cuda_check(cudaMemcpyAsync(drank.b.p, trank.data(), (size_t)ntask * 4,
                                                 cudaMemcpyHostToDevice, s), "rank upload")))
                return rc;
            if ((rc = cuda_check(cudaMemcpyAsync(doff.b.p, toff.data(), (size_t)ntask * 8,
                                                 cudaMemcpyHostToDevice, s), "offset upload")))
                return rc;
            HM_CUDA(cudaStreamSynchronize(s));
            for (int32_t f : ff)
                if (f & 8) return fail(HM_EDEVICE, "ACA factor arena overflow on re-run");
        }
    }
    HM_CUDA(cudaEventRecord(ev[2], s));

    // ---- block-ordered FP64 factor arenas
    for (int64_t q = 0; q < ntask; ++q) {
        const AcaTask& tk = tasks[(size_t)q];
        const Blk& b = H.adm_h[(size_t)tk.blk];
        H.rank_h[(size_t)(tk.blk * 7 + tk.kern)] = trank[(size_t)q];
        // bit 0: the sequence reached the rank cap below min(|t|, |s|)
        H.flags_h[(size_t)(tk.blk * 7 + tk.kern)] =
            tflags[(size_t)q] | (trank[(size_t)q] >= H.prm.kmax && H.prm.kmax < std::min(b.m, b.n) ? 1 : 0);
    }
    const int64_t nbk = H.nadm * 7;
    H.uoff_h.resize((size_t)nbk);
    H.voff_h.resize((size_t)nbk);
    H.coff_h.resize((size_t)nbk);
    int64_t ut = 0, vt = 0, ct = 0;
    for (int64_t b = 0; b < H.nadm; ++b)
        for (int k = 0; k < 7; ++k) {
            size_t q = (size_t)(b * 7 + k);
            int32_t r = H.rank_h[q];
            const Blk& bk = H.adm_h[(size_t)b];
            H.uoff_h[q] = ut;
            H.voff_h[q] = vt;
            H.coff_h[q] = ct;
            // keep every factor start 16-byte aligned for vector loads
            ut += ((int64_t)r * bk.m + 7) & ~int64_t(7);
            vt += ((int64_t)r * bk.n + 7) & ~int64_t(7);
            ct += r;
        }
    H.u_total = ut;
    H.v_total = vt;
    H.c_total = ct;
    H.w_total = 4 * ct;  // w holds one 4-vector per factor column
    if ((rc = dalloc(H, H.U64, (size_t)std::max<int64_t>(ut, 1) * 8))) return rc;
    if ((rc = dalloc(H, H.V64, (size_t)std::max<int64_t>(vt, 1) * 8))) return rc;
    if ((rc = upload(H, H.d_uoff, H.uoff_h.data(), (size_t)nbk * 8))) return rc;
    if ((rc = upload(H, H.d_voff, H.voff_h.data(), (size_t)nbk * 8))) return rc;
    if ((rc = upload(H, H.d_coff, H.coff_h.data(), (size_t)nbk * 8))) return rc;
    if ((rc = upload(H, H.d_rank, H.rank_h.data(), (size_t)nbk * 4))) return rc;
    if (ntask > 0) {
        repack_kernel<<<(unsigned)ntask, 128, 0, s>>>(
            dtask.b.as<AcaTask>(), (int)ntask, H.d_adm.as<Blk>(), drank.b.as<int32_t>(),
            doff.b.as<int64_t>(), darena.b.as<double>(), (int64_t)cap, darena2.b.as<double>(), H.d_uoff.as<int64_t>(),
            H.d_voff.as<int64_t>(), H.U64.as<double>(), H.V64.as<double>());
        HM_CUDA(cudaGetLastError());
    }
    HM_CUDA(cudaEventRecord(ev[3], s));

    // ---- streaming layouts of the product (element offsets; the arenas of
    // each form are filled by pack_device)
    //   U, per leaf tau: for every admissible block t x s with t containing
    //     tau (root first) and every kernel with k > 0, the k columns of
    //     U[rows of tau, :] as segments of mp = roundup(|tau|, 8) elements;
    //   near field, per leaf: for every near block tau x sigma and column j,
    //     six segments (V_11, V_12, V_13, V_22, V_23, V_33) of mp elements;
    //   V, per admissible block: row-major |s| x Cp, Cp = roundup(sum k, 8).
    {
        std::vector<std::vector<int32_t>> adm_by_row(tr.nodes.size()), near_by_row(tr.nodes.size());
        for (int64_t b = 0; b < H.nadm; ++b) adm_by_row[(size_t)tr.adm[(size_t)b][0]].push_back((int32_t)b);
        for (int64_t b = 0; b < H.nnear; ++b)
            near_by_row[(size_t)tr.near_blocks[(size_t)b][0]].push_back((int32_t)b);
        int32_t csp = 0;
        for (size_t n = 0; n < tr.nodes.size(); ++n)
            csp = std::max<int32_t>(csp, (int32_t)(adm_by_row[n].size() + near_by_row[n].size()));
        H.csp = csp;
        std::vector<int64_t> parent(tr.nodes.size(), -1);
        for (size_t n = 0; n < tr.nodes.size(); ++n)
            for (int c = 0; c < 2; ++c)
                if (tr.nodes[n].son[c] >= 0) parent[(size_t)tr.nodes[n].son[c]] = (int64_t)n;
        std::vector<int32_t> leafv, lf_ptr(1, 0), ln_ptr(1, 0);
        std::vector<int64_t> lf_base, ln_base;
        std::vector<LeafFarItem> lf_items, lr_items;
        std::vector<int32_t> lr_ptr(1, 0);
        std::vector<PackSrc> lf_src;
        std::vector<LeafNearItem> ln_items;
        std::vector<NearSrc> ln_src;
        std::vector<int64_t> ln16_base;   // byte offsets in the INT16 near stream
        std::vector<int32_t> ln16_diag;   // columns of the leaf's diagonal block
        int64_t ul = 0, nl = 0, nl16 = 0, nl_diag = 0;
        int32_t maxleaf = 0;
        for (int64_t lf : tr.leaves) {
            const Node& L = tr.nodes[(size_t)lf];
            const int32_t mt = (int32_t)(L.hi - L.lo);
            const int64_t mp = (mt + 7) & ~7;
            leafv.push_back((int32_t)L.lo);
            leafv.push_back(mt);
            maxleaf = std::max(maxleaf, mt);
            std::vector<int64_t> chain;
            for (int64_t n = lf; n >= 0; n = parent[(size_t)n]) chain.push_back(n);
            std::reverse(chain.begin(), chain.end());  // root first
            int32_t seg = 0;
            lf_base.push_back(ul);
            for (int64_t n : chain)
                for (int32_t b : adm_by_row[(size_t)n]) {
                    const int32_t off = (int32_t)(L.lo - tr.nodes[(size_t)n].lo);
                    for (int k = 0; k < 7; ++k) {
                        const size_t q = (size_t)b * 7 + k;
                        const int32_t r = H.rank_h[q];
                        if (r == 0) continue;
                        lf_items.push_back(LeafFarItem{seg, (int32_t)H.coff_h[q]});
                        lf_src.push_back(PackSrc{H.uoff_h[q] + off, H.adm_h[(size_t)b].m, r});
                        seg += r;
                    }
                }
            lf_items.push_back(LeafFarItem{seg, 0});  // sentinel: number of segments
            lf_src.push_back(PackSrc{0, 0, 0});
            // w runs: an item continues the previous run when its columns do
            for (int32_t q = lf_ptr.back(); q + 1 < (int32_t)lf_items.size(); ++q) {
                const LeafFarItem it = lf_items[(size_t)q];
                if (q > lf_ptr.back()) {
                    const LeafFarItem& pv = lf_items[(size_t)q - 1];
                    if (it.col == pv.col + (it.seg_start - pv.seg_start)) continue;
                }
                lr_items.push_back(it);
            }
            lr_items.push_back(LeafFarItem{seg, 0});
            lr_ptr.push_back((int32_t)lr_items.size());
            lf_ptr.push_back((int32_t)lf_items.size());
            // the 16-bit forms take segments 16 at a time (one tensor-core K step):
            // every leaf's U stream holds a multiple of 16 segments, zero padded
            ul += (int64_t)((seg + 15) & ~15) * mp;
            int32_t col = 0;
            ln_base.push_back(nl);
            // the leaf's diagonal block (tau, tau) first: it holds the singular
            // and near-singular pairs, which the INT16 form keeps in FP32
            std::vector<int32_t> nb_order(near_by_row[(size_t)lf].begin(), near_by_row[(size_t)lf].end());
            std::stable_partition(nb_order.begin(), nb_order.end(), [&](int32_t b) {
                return H.near_h[(size_t)b].s0 == (int32_t)L.lo && H.near_h[(size_t)b].n == mt;
            });
            int32_t ndiag = 0;
            for (int32_t b : nb_order) {
                const Blk& bk = H.near_h[(size_t)b];
                if (col == 0 && bk.s0 == (int32_t)L.lo && bk.n == mt) ndiag = bk.n;
                ln_items.push_back(LeafNearItem{col, bk.s0});
                ln_src.push_back(NearSrc{H.noff_h[(size_t)b], bk.n, 0});
                col += bk.n;
            }
            ln_items.push_back(LeafNearItem{col, 0});  // sentinel: number of columns
            ln_src.push_back(NearSrc{0, 0, 0});
            ln_ptr.push_back((int32_t)ln_items.size());
            nl += (int64_t)col * 6 * mp;
            // the INT16 near stream: the columns after the diagonal block, each a
            // 32-byte header (six FP32 scales) and six segments of mp int16
            ln16_base.push_back(nl16);
            ln16_diag.push_back(ndiag);
            nl_diag += (int64_t)ndiag * 6 * mp;
            nl16 += (int64_t)(col - ndiag) * (kNear16Head + 12 * mp);
        }
        H.max_leaf = maxleaf;
        H.ul_total = ul;
        H.nl_total = nl;
        H.nl16_bytes = nl16;
        H.nl_diag_total = nl_diag;
        H.nleaves = (int64_t)tr.leaves.size();
        {
            // streamed kernel: leaves with the most bytes first
            std::vector<int64_t> bytes(tr.leaves.size());
            for (size_t l = 0; l < tr.leaves.size(); ++l) {
                const int64_t mp = (leafv[2 * l + 1] + 7) & ~7;
                bytes[l] = (int64_t)lf_items[(size_t)lf_ptr[l + 1] - 1].seg_start * mp +
                           (int64_t)ln_items[(size_t)ln_ptr[l + 1] - 1].col_start * 6 * mp;
            }
            std::vector<int32_t> order(tr.leaves.size());
            std::iota(order.begin(), order.end(), 0);
            std::stable_sort(order.begin(), order.end(),
                             [&](int32_t a, int32_t b) { return bytes[(size_t)a] > bytes[(size_t)b]; });
            std::vector<int2> work(order.size());
            for (size_t q = 0; q < order.size(); ++q) work[q] = make_int2(0, order[q]);
            H.leaf_order_h = order;
            H.leaf_bytes_h = bytes;
            if ((rc = upload(H, H.d_work, work.data(), work.size() * sizeof(int2)))) return rc;
            const int64_t pp[2] = {0, M};
            if ((rc = upload(H, H.d_pos_prefix, pp, sizeof pp))) return rc;
        }
        if ((rc = upload(H, H.d_leaf, leafv.data(), leafv.size() * 4))) return rc;
        if ((rc = upload(H, H.d_lf_base, lf_base.data(), lf_base.size() * 8))) return rc;
        if ((rc = upload(H, H.d_lf_ptr, lf_ptr.data(), lf_ptr.size() * 4))) return rc;
        if ((rc = upload(H, H.d_lf_items, lf_items.data(), lf_items.size() * sizeof(LeafFarItem)))) return rc;
        if ((rc = upload(H, H.d_lr_ptr, lr_ptr.data(), lr_ptr.size() * 4))) return rc;
        if ((rc = upload(H, H.d_lr_items, lr_items.data(), lr_items.size() * sizeof(LeafFarItem)))) return rc;
        if ((rc = upload(H, H.d_lf_src, lf_src.data(), lf_src.size() * sizeof(PackSrc)))) return rc;
        if ((rc = upload(H, H.d_ln_base, ln_base.data(), ln_base.size() * 8))) return rc;
        if ((rc = upload(H, H.d_ln_ptr, ln_ptr.data(), ln_ptr.size() * 4))) return rc;
        if ((rc = upload(H, H.d_ln_items, ln_items.data(), ln_items.size() * sizeof(LeafNearItem)))) return rc;
        if ((rc = upload(H, H.d_ln_src, ln_src.data(), ln_src.size() * sizeof(NearSrc)))) return rc;
        if ((rc = upload(H, H.d_ln16_base, ln16_base.data(), ln16_base.size() * 8))) return rc;
        if ((rc = upload(H, H.d_ln16_diag, ln16_diag.data(), ln16_diag.size() * 4))) return rc;
    }
    {
        // forward-pass groups: the admissible blocks that share a column
        // cluster s (at most kMaxGroupRecs each) store their row-major V side
        // by side, one |s| x Cs matrix per group (block b's Cp_b = sum of its
        // ranks rounded up to 8 columns at column offset coff_b), so that the
        // forward pass reads x(s) once per group; groups with the most data
        // first
        std::vector<std::vector<int32_t>> by_col(tr.nodes.size());
        for (int64_t b = 0; b < H.nadm; ++b) {
            int32_t Csum = 0;
            for (int k = 0; k < 7; ++k) Csum += H.rank_h[(size_t)(b * 7 + k)];
            if (Csum > 0) by_col[(size_t)tr.adm[(size_t)b][1]].push_back((int32_t)b);
        }
        struct G0 {
            int64_t work;
            std::vector<int32_t> blocks;
        };
        std::vector<G0> gl;
        for (size_t nd = 0; nd < tr.nodes.size(); ++nd) {
            const auto& L = by_col[nd];
            for (size_t i0 = 0; i0 < L.size(); i0 += kMaxGroupRecs) {
                G0 g;
                g.blocks.assign(L.begin() + (int64_t)i0, L.begin() + (int64_t)std::min(L.size(), i0 + kMaxGroupRecs));
                g.work = 0;
                for (int32_t b : g.blocks)
                    for (int k = 0; k < 7; ++k)
                        g.work += (int64_t)H.rank_h[(size_t)(b * 7 + k)] * H.adm_h[(size_t)b].n;
                gl.push_back(std::move(g));
            }
        }
        std::stable_sort(gl.begin(), gl.end(), [](const G0& a, const G0& b) { return a.work > b.work; });
        std::vector<int64_t> vb_base((size_t)H.nadm + 1, 0), vb_ld((size_t)H.nadm + 1, 0),
            vb_coff((size_t)H.nadm + 1, 0);
        std::vector<FwdRec> recs;
        std::vector<FwdGroup> groups;
        int64_t vr = 0, dcols = 0;
        for (const G0& g0 : gl) {
            FwdGroup g{};
            const Blk& b0 = H.adm_h[(size_t)g0.blocks[0]];
            g.vbase = vr;
            g.s0 = b0.s0;
            g.n = b0.n;
            g.first = (int32_t)recs.size();
            g.nrec = (int16_t)g0.blocks.size();
            g.mesh = 0;
            int64_t cs = 0;
            for (int32_t b : g0.blocks) {
                FwdRec r{};
                const Blk& bk = H.adm_h[(size_t)b];
                r.s0 = bk.s0;
                r.n = bk.n;
                r.col0 = (int32_t)H.coff_h[(size_t)b * 7];
                r.mesh = 0;
                int32_t Csum = 0;
                for (int k = 0; k < 7; ++k) {
                    const int32_t kk = H.rank_h[(size_t)(b * 7 + k)];
                    if (kk > 255) return fail(HM_EINVAL, "rank %d above 255 is not supported", kk);
                    r.kpack |= (uint64_t)kk << (8 * k);
                    Csum += kk;
                }
                r.C = (int16_t)Csum;
                r.coff = (int32_t)cs;  // column offset in the group
                r.grp = (int32_t)groups.size();
                vb_base[(size_t)b] = vr;
                vb_coff[(size_t)b] = cs;
                cs += (Csum + 7) & ~7;
                recs.push_back(r);
            }
            if (cs > INT32_MAX / 8) return fail(HM_EINVAL, "forward group too wide");
            g.Cs = (int32_t)cs;
            if (dcols + cs > INT32_MAX) return fail(HM_EINVAL, "too many forward-group columns");
            g.dbase = (int32_t)dcols;
            dcols += cs;
            for (int32_t b : g0.blocks) vb_ld[(size_t)b] = cs;
            // rows padded to 16 (a tensor-core K step; the 16-bit forms store V
            // in 8 x 8 tiles, see pack_vr_kernel)
            vr += (int64_t)((g.n + 15) & ~15) * cs;
            groups.push_back(g);
        }
        vb_base[(size_t)H.nadm] = vr;
        H.vr_total = vr;
        H.dcols = dcols;
        // units: one CTA per kFwdUnitRows rows of a group, the most data first
        std::vector<FwdUnit> units;
        std::vector<FwdMulti> multi;
        int64_t zc = 0;
        for (size_t gi = 0; gi < groups.size(); ++gi) {
            const FwdGroup& g = groups[gi];
            const int32_t nch = (g.n + kFwdUnitRows - 1) / kFwdUnitRows;
            const int64_t z0 = nch > 1 ? zc : -1;
            if (nch > 1) {
                for (int32_t c0 = 0; c0 < g.Cs; c0 += kReduceCols)
                    multi.push_back(FwdMulti{(int32_t)gi, nch, zc, c0, std::min(kReduceCols, g.Cs - c0)});
                zc += (int64_t)nch * g.Cs;
            }
            for (int32_t k = 0; k < nch; ++k)
                for (int32_t c0 = 0; c0 < g.Cs; c0 += kFwdUnitCols)
                    units.push_back(FwdUnit{(int32_t)gi, k * kFwdUnitRows, std::min(kFwdUnitRows, g.n - k * kFwdUnitRows),
                                            k, c0, std::min(kFwdUnitCols, g.Cs - c0), z0});
        }
        std::stable_sort(units.begin(), units.end(), [&](const FwdUnit& a, const FwdUnit& b) {
            return (int64_t)a.nrows * a.ncols > (int64_t)b.nrows * b.ncols;
        });
        H.zcols = zc;
        H.unit_h = units;
        H.multi_h = multi;
        H.fwd_h = recs;
        H.grp_h = groups;
        // per-block lists for the several-vector forward kernels
        std::vector<int32_t> bigv, smallv;
        {
            std::vector<int32_t> ord(recs.size());
            std::iota(ord.begin(), ord.end(), 0);
            std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
                return (int64_t)recs[(size_t)a].n * recs[(size_t)a].C > (int64_t)recs[(size_t)b].n * recs[(size_t)b].C;
            });
            for (int32_t q : ord) (recs[(size_t)q].n > 128 ? bigv : smallv).push_back(q);
        }
        H.big_h = bigv;
        H.small_h = smallv;
        if ((rc = upload(H, H.d_big, bigv.data(), bigv.size() * 4))) return rc;
        if ((rc = upload(H, H.d_small, smallv.data(), smallv.size() * 4))) return rc;
        if ((rc = upload(H, H.d_units, units.data(), units.size() * sizeof(FwdUnit)))) return rc;
        {
            const std::vector<FwdTcUnit> tcu = tc_units(units, groups);
            if ((rc = upload(H, H.d_tcunits, tcu.data(), tcu.size() * sizeof(FwdTcUnit)))) return rc;
        }
        if ((rc = upload(H, H.d_multi, multi.data(), multi.size() * sizeof(FwdMulti)))) return rc;
        if ((rc = upload(H, H.d_fwd_all, recs.data(), recs.size() * sizeof(FwdRec)))) return rc;
        if ((rc = upload(H, H.d_groups, groups.data(), groups.size() * sizeof(FwdGroup)))) return rc;
        if ((rc = upload(H, H.d_vb_base, vb_base.data(), vb_base.size() * 8))) return rc;
        if ((rc = upload(H, H.d_vb_ld, vb_ld.data(), vb_ld.size() * 8))) return rc;
        if ((rc = upload(H, H.d_vb_coff, vb_coff.data(), vb_coff.size() * 8))) return rc;
        if (H.c_total > INT32_MAX / 4) return fail(HM_EINVAL, "too many factor columns");
    }
    // ---- workspace for the product
    H.max_rhs = H.prm.max_rhs;
    if ((rc = dalloc(H, H.xg, (size_t)H.max_rhs * 4 * M * 8))) return rc;
    if ((rc = dalloc(H, H.wb, (size_t)H.max_rhs * std::max<int64_t>(H.w_total, 1) * 8))) return rc;
    if ((rc = dalloc(H, H.zb, (size_t)H.max_rhs * std::max<int64_t>(H.zcols, 1) * 4 * 8))) return rc;
    if ((rc = dalloc(H, H.d_counters, (size_t)kCounterInts * sizeof(int)))) return rc;
    if ((rc = dalloc(H, H.d_err, 64))) return rc;
    HM_CUDA(cudaMemsetAsync(H.d_err.p, 0, 64, s));

    if ((rc = dalloc(H, H.xh, (size_t)H.max_rhs * 3 * M * 8))) return rc;
    if ((rc = dalloc(H, H.yh, (size_t)H.max_rhs * 3 * M * 8))) return rc;
    // the FP64 form, unless deferred to hm_pack
    if (!(H.prm.flags & (HM_DEFER_FP64 | HM_DEFER_ACA)))
        if ((rc = pack_device(H, HM_FP64, s))) return rc;
    HM_CUDA(cudaStreamSynchronize(s));
    float t01 = 0, t12 = 0, t23 = 0;
    cudaEventElapsedTime(&t01, ev[0], ev[1]);
    cudaEventElapsedTime(&t12, ev[1], ev[2]);
    cudaEventElapsedTime(&t23, ev[2], ev[3]);
    {
        unsigned long long cnt[5] = {0, 0, 0, 0, 0};
        HM_CUDA(cudaMemcpy(cnt, qc, sizeof cnt, cudaMemcpyDeviceToHost));
        for (int i = 0; i < 5; ++i) H.asm_count[i] = (int64_t)cnt[i];
    }
    H.asm_ms[0] = t01;
    H.asm_ms[1] = t12 + t23;
    H.asm_ms[2] = 0.0;
    return HM_OK;
}

// The evaluation operator ~V_h of Section 5, Eq. (vector_eq): rows are the
// points of `tr` (a point tree), columns the triangles of tr.src.  The same
// entries with the point in place of a centroid (never a self pair), the near
// blocks entry by entry and Algorithm 1 on every admissible block and kernel
// (run as one batched launch per size class, with an exact arena bound), the
// factors then copied to block order.  No packed forms: the product is the
// exact FP64 one of hm_eval_points (and the adaptive one of hm_amvm).
int assemble_points_device(const hm_tree& tr, hm_matrix& H)
{
    cudaStream_t s = H.alloc.stream;
    const hm_tree& src = *tr.src;
    // kind 1: rows the points of tr, columns the triangles of src (~V_h);
    // kind 2: rows the triangles of src, columns the vertices of tr (K_Delta)
    const bool dl = tr.kind == 2;
    const std::vector<Node>& rnodes = dl ? src.nodes : tr.nodes;
    const std::vector<Node>& cnodes = dl ? tr.nodes : src.nodes;
    const int64_t M = dl ? tr.M : src.M, Mr = dl ? src.M : tr.M;
    H.M = M;
    H.Mr = Mr;
    H.rect = true;
    H.dl = dl;
    H.mesh_fp = mesh_fingerprint(src);
    H.nleaves = (int64_t)(dl ? src.leaves.size() : tr.leaves.size());
    int rc;
    if ((rc = upload_tables(s))) return rc;
    if ((rc = upload_geometry(src, H))) return rc;
    if (!dl) {
        std::vector<int32_t> rperm((size_t)Mr);
        std::vector<double> rows((size_t)(3 * Mr));
        for (int64_t p = 0; p < Mr; ++p) {
            const int64_t i = tr.perm[(size_t)p];
            rperm[(size_t)p] = (int32_t)i;
            for (int k = 0; k < 3; ++k) rows[(size_t)(3 * p + k)] = tr.coll[(size_t)(3 * i + k)];
        }
        if ((rc = upload(H, H.d_rperm, rperm.data(), rperm.size() * 4))) return rc;
        if ((rc = upload(H, H.g_rows, rows.data(), rows.size() * 8))) return rc;
    } else if ((rc = upload_dl_geometry(tr, H))) {
        return rc;
    }
    Geom g{H.g_coll.as<double>(), H.g_tri.as<double>(), H.g_qp.as<double>(), H.g_qw.as<double>(),
           H.g_diam.as<double>(), H.g_rows.as<double>(), 0};
    if (dl) {
        g.nrm = H.g_nrm.as<double>();
        g.star_ptr = H.d_star_ptr.as<int32_t>();
        g.star = H.d_star.as<int32_t>();
    }

    // ---- block lists: (row node, column node) of the partition
    auto blk_of = [&](const std::array<int64_t, 2>& ts) {
        const Node& a = rnodes[(size_t)ts[0]];
        const Node& c = cnodes[(size_t)ts[1]];
        return Blk{(int32_t)a.lo, (int32_t)(a.hi - a.lo), (int32_t)c.lo, (int32_t)(c.hi - c.lo)};
    };
    H.nadm = (int64_t)tr.adm.size();
    H.nnear = (int64_t)tr.near_blocks.size();
    H.adm_h.resize((size_t)H.nadm);
    H.near_h.resize((size_t)H.nnear);
    for (int64_t b = 0; b < H.nadm; ++b) H.adm_h[(size_t)b] = blk_of(tr.adm[(size_t)b]);
    for (int64_t b = 0; b < H.nnear; ++b) H.near_h[(size_t)b] = blk_of(tr.near_blocks[(size_t)b]);
    if ((rc = upload(H, H.d_adm, H.adm_h.data(), H.adm_h.size() * sizeof(Blk)))) return rc;
    if ((rc = upload(H, H.d_near, H.near_h.data(), H.near_h.size() * sizeof(Blk)))) return rc;
    {
        // c_sp (Section 2.1): the most blocks sharing a row or a column cluster
        std::vector<int32_t> rc_cnt(rnodes.size(), 0), cc_cnt(cnodes.size(), 0);
        int32_t csp = 0;
        for (const auto* L : {&tr.adm, &tr.near_blocks})
            for (const auto& ts : *L) {
                csp = std::max(csp, ++rc_cnt[(size_t)ts[0]]);
                csp = std::max(csp, ++cc_cnt[(size_t)ts[1]]);
            }
        H.csp = csp;
    }

    cudaEvent_t ev[4];
    for (auto& e : ev) HM_CUDA(cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t* e;
        ~EvGuard()
        {
            for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]);
        }
    } evg{ev};

    // ---- near field
    H.noff_h.resize((size_t)H.nnear);
    int64_t ntot = 0;
    for (int64_t b = 0; b < H.nnear; ++b) {
        H.noff_h[(size_t)b] = ntot;
        ntot += 6 * (int64_t)H.near_h[(size_t)b].m * H.near_h[(size_t)b].n;
    }
    H.n_total = ntot;
    if ((rc = upload(H, H.d_noff, H.noff_h.data(), H.noff_h.size() * 8))) return rc;
    if ((rc = dalloc(H, H.N64, (size_t)std::max<int64_t>(ntot, 1) * 8))) return rc;
    HM_CUDA(cudaEventRecord(ev[0], s));
    if (H.nnear > 0) {
        if (dl)
            dl_near_kernel<<<(unsigned)H.nnear, 128, 0, s>>>(g, H.d_near.as<Blk>(), H.d_noff.as<int64_t>(),
                                                             H.N64.as<double>());
        else
            near_kernel<<<(unsigned)H.nnear, 128, 0, s>>>(g, H.d_near.as<Blk>(), H.d_noff.as<int64_t>(),
                                                          H.N64.as<double>(), nullptr);
        HM_CUDA(cudaGetLastError());
    }
    HM_CUDA(cudaEventRecord(ev[1], s));

    // ---- Algorithm 1 on every admissible block and kernel that does not
    // vanish identically (as for the square matrix: every point and source
    // point of the block shares coordinate a)
    const int64_t nbk = H.nadm * 7;
    H.rank_h.assign((size_t)nbk, 0);
    H.flags_h.assign((size_t)nbk, 0);
    static const int kp[7] = {-1, 0, 0, 0, 1, 1, 2}, kq[7] = {-1, 0, 1, 2, 1, 2, 2};
    std::vector<int32_t> bk;
    for (int64_t b = 0; b < H.nadm; ++b) {
        if (dl) {
            // K_Delta is one scalar kernel: slot 0 (the other six keep rank 0)
            bk.push_back((int32_t)(b * 7));
            continue;
        }
        const Node& nt = tr.nodes[(size_t)tr.adm[(size_t)b][0]];
        const Node& ns = src.nodes[(size_t)tr.adm[(size_t)b][1]];
        for (int k = 0; k < 7; ++k) {
            bool zero = false;
            if (k > 0)
                for (int a : {kp[k], kq[k]})
                    if (nt.bmin[a] == nt.bmax[a] && ns.bmin[a] == ns.bmax[a] && nt.bmin[a] == ns.bmin[a])
                        zero = true;
            if (zero)
                H.flags_h[(size_t)(b * 7 + k)] = 32;
            else
                bk.push_back((int32_t)(b * 7 + k));
        }
    }
    if (H.prm.flags & HM_DEFER_ACA) {
        bk.clear();
        H.aca_deferred = true;
    }
    DevBuf arena;
    struct ArenaGuard {
        hm_matrix& H;
        DevBuf& a;
        ~ArenaGuard() { H.alloc.release(a.p, a.bytes); }
    } ag{H, arena};
    std::vector<int32_t> trank, tflags;
    std::vector<int64_t> toff;
    size_t hint = 0;
    {
        // first arena: rank 12 per block and kernel (the measured means are
        // 7-11 at eps 1e-4 .. 1e-8), at most 60% of the free device memory;
        // a batch that does not fit runs again into an arena of the exact size
        double est = 1.0;
        for (int32_t v : bk) {
            const Blk& b = H.adm_h[(size_t)(v / 7)];
            est += (double)(b.m + b.n) * std::min(12, std::min(b.m, b.n));
        }
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) est = std::min(est, 0.6 * (double)fr / 8.0 / 1.1);
        else cudaGetLastError();
        hint = (size_t)(est * 1.1) + (size_t(1) << 20);
    }
    if ((rc = aca_on_demand(H, bk, H.prm.kmax, s, arena, trank, toff, nullptr, &tflags, hint))) return rc;
    HM_CUDA(cudaEventRecord(ev[2], s));
    for (size_t q = 0; q < bk.size(); ++q) {
        H.rank_h[(size_t)bk[q]] = trank[q];
        // bit 0: the sequence reached the rank cap below min(|t|, |s|)
        const Blk& b = H.adm_h[(size_t)(bk[q] / 7)];
        H.flags_h[(size_t)bk[q]] = tflags[q] | (trank[q] >= H.prm.kmax && H.prm.kmax < std::min(b.m, b.n) ? 1 : 0);
    }

    // ---- block-ordered FP64 factor arenas
    H.uoff_h.resize((size_t)nbk);
    H.voff_h.resize((size_t)nbk);
    H.coff_h.resize((size_t)nbk);
    int64_t ut = 0, vt = 0, ct = 0;
    for (int64_t b = 0; b < H.nadm; ++b)
        for (int k = 0; k < 7; ++k) {
            const size_t q = (size_t)(b * 7 + k);
            const int32_t r = H.rank_h[q];
            const Blk& bb = H.adm_h[(size_t)b];
            H.uoff_h[q] = ut;
            H.voff_h[q] = vt;
            H.coff_h[q] = ct;
            ut += ((int64_t)r * bb.m + 7) & ~int64_t(7);
            vt += ((int64_t)r * bb.n + 7) & ~int64_t(7);
            ct += r;
        }
    H.u_total = ut;
    H.v_total = vt;
    H.c_total = ct;
    if ((rc = dalloc(H, H.U64, (size_t)std::max<int64_t>(ut, 1) * 8))) return rc;
    if ((rc = dalloc(H, H.V64, (size_t)std::max<int64_t>(vt, 1) * 8))) return rc;
    if ((rc = upload(H, H.d_uoff, H.uoff_h.data(), (size_t)nbk * 8))) return rc;
    if ((rc = upload(H, H.d_voff, H.voff_h.data(), (size_t)nbk * 8))) return rc;
    if ((rc = upload(H, H.d_coff, H.coff_h.data(), (size_t)nbk * 8))) return rc;
    if ((rc = upload(H, H.d_rank, H.rank_h.data(), (size_t)nbk * 4))) return rc;
    if (!bk.empty()) {
        std::vector<AcaTask> tasks(bk.size());
        for (size_t q = 0; q < bk.size(); ++q) tasks[q] = AcaTask{bk[q] / 7, bk[q] % 7};
        TmpBuf dtask(H), drank(H), doff(H);
        if ((rc = upload(H, dtask.b, tasks.data(), tasks.size() * sizeof(AcaTask)))) return rc;
        if ((rc = upload(H, drank.b, trank.data(), trank.size() * 4))) return rc;
        if ((rc = upload(H, doff.b, toff.data(), toff.size() * 8))) return rc;
        // every offset lies in the one arena (cap = its size)
        repack_kernel<<<(unsigned)bk.size(), 128, 0, s>>>(
            dtask.b.as<AcaTask>(), (int)bk.size(), H.d_adm.as<Blk>(), drank.b.as<int32_t>(), doff.b.as<int64_t>(),
            arena.as<double>(), (int64_t)(arena.bytes / 8), arena.as<double>(), H.d_uoff.as<int64_t>(),
            H.d_voff.as<int64_t>(), H.U64.as<double>(), H.V64.as<double>());
        HM_CUDA(cudaGetLastError());
        HM_CUDA(cudaStreamSynchronize(s));
    }
    HM_CUDA(cudaEventRecord(ev[3], s));
    H.max_rhs = H.prm.max_rhs;
    if ((rc = dalloc(H, H.d_err, 64))) return rc;
    HM_CUDA(cudaMemsetAsync(H.d_err.p, 0, 64, s));
    if ((rc = eval_prepare(H))) return rc;
    HM_CUDA(cudaStreamSynchronize(s));
    float t01 = 0, t12 = 0, t23 = 0;
    cudaEventElapsedTime(&t01, ev[0], ev[1]);
    cudaEventElapsedTime(&t12, ev[1], ev[2]);
    cudaEventElapsedTime(&t23, ev[2], ev[3]);
    H.asm_ms[0] = t01;
    H.asm_ms[1] = t12 + t23;
    H.asm_ms[2] = 0.0;
    return HM_OK;
}

}  // namespace hm

extern "C" int hm_aca_assemble(const hm_tree* tree, const hm_params* prm, const hm_allocator* alloc,
                               void* stream, hm_matrix** out)
{
    using namespace hm;
    if (!out) return fail(HM_EINVAL, "hm_aca_assemble: out is NULL");
    *out = nullptr;
    if (!tree || !prm) return fail(HM_EINVAL, "hm_aca_assemble: NULL tree or params");
    if (!(prm->E > 0.0) || !std::isfinite(prm->E)) return fail(HM_EINVAL, "hm_aca_assemble: E must be > 0");
    if (!(prm->nu > 0.0 && prm->nu < 0.5)) return fail(HM_EINVAL, "hm_aca_assemble: nu must lie in (0, 1/2)");
    if (!(prm->aca_eps > 0.0) || !(prm->aca_eps < 1.0))
        return fail(HM_EINVAL, "hm_aca_assemble: aca_eps must lie in (0, 1)");
    if (!(prm->aca_eta_stop >= 0.0 && prm->aca_eta_stop < 1.0))
        return fail(HM_EINVAL, "hm_aca_assemble: aca_eta_stop must lie in [0, 1)");
    if (prm->kmax < 0 || prm->kmax > kKmaxLimit)
        return fail(HM_EINVAL, "hm_aca_assemble: kmax must lie in 0..%d", kKmaxLimit);
    if (prm->max_rhs < 0 || prm->max_rhs > 64) return fail(HM_EINVAL, "hm_aca_assemble: max_rhs must lie in 0..64");
    if (prm->flags & ~(HM_DEFER_FP64 | HM_DEFER_ACA))
        return fail(HM_EINVAL, "hm_aca_assemble: unknown flags 0x%x", prm->flags);
    hm_matrix* H = new (std::nothrow) hm_matrix();
    if (!H) return fail(HM_ENOMEM, "hm_aca_assemble: out of host memory");
    H->prm = *prm;
    if (H->prm.kmax == 0) H->prm.kmax = 128;
    if (H->prm.max_rhs == 0) H->prm.max_rhs = 32;
    H->E = prm->E;
    H->nu = prm->nu;
    H->alloc.stream = (cudaStream_t)stream;
    if (alloc && alloc->alloc && alloc->free) {
        H->alloc.user = *alloc;
        H->alloc.has_user = true;
    }
    int rc;
    try {
        rc = assemble_device(*tree, *H);
    } catch (const std::bad_alloc&) {
        rc = fail(HM_ENOMEM, "hm_aca_assemble: out of host memory");
    }
    if (rc) {
        hm_matrix_destroy(H);
        return rc;
    }
    *out = H;
    for (int32_t f : H->flags_h)
        if (f & 1) {
            set_error("hm_aca_assemble: a block reached the rank cap kmax=%d", H->prm.kmax);
            return HM_ERANK;
        }
    return HM_OK;
}
