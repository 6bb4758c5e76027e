/*
 * hm_oracle.c -- plain, slow, FP64 CPU oracle for the collocation Lame
 * single-layer H-matrix (Bauer & Bebendorf, "Adaptive H-Matrix Computations in
 * Linear Elasticity").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the CUDA
 * library.  Compile with -ffp-contract=off so that every product and sum is
 * rounded separately, in the order written here.
 *
 * What each part follows:
 *   Kelvin tensor                  Section 4.1, definition of S_K
 *   scalar kernels V_Delta, V_kl   Section 4.2, Eq. (Vh) (prefactor read as 1/(4 pi))
 *   collocation at centroids       Section 2, collocation example (Lambda_1 f)_i = f(y_i)
 *   cluster tree                   Section 2.1 (binary, disjoint sons, leaves of size <= b_min)
 *   admissibility / partition      Section 2.1, Eq. (adm) and the block-cluster recursion
 *   ACA                            Section 2.2, Algorithm 1 and the cross representation after it
 *   H-matrix-vector product        Section 2 (O(k(M+N)) product of a low-rank block) and Section 2.2
 *   double layer K_h               Section 4.2, Eq. (Kh) (K_Delta with hat functions, the surface curls
 *                                  T_h, V_Delta T_h and V_h T_h; collocation at the centroids)
 *   evaluation operator ~V_h       Section 5, Eq. (vector_eq) (u_h at points x_i of the domain: the collocation
 *                                  entries with x_i for the centroid; a tree of the points)
 *
 * Quadrature contract (the paper names no rule; this is the reading both the
 * oracle and the CUDA path implement):
 *   self pair (j == i): tau_i split at c_i into three sub-triangles, Duffy map
 *     collapsing the apex; the radial integral is exact and the remaining 1-D
 *     integral uses n_D = 32 Gauss-Legendre points per sub-triangle;
 *   other pairs: recursive 4-way midpoint subdivision of tau_j while
 *     |x - g(sub)|^2 < rho^2 diam(sub)^2 (rho = 2, depth < 8), Radon's 7-point
 *     degree-5 rule on every leaf; a well-separated pair is a leaf at depth 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_RHO2 4.0
#define OR_MAXDEPTH 8
#define OR_ND 32

/* ------------------------------------------------------------------------ */
/* Quadrature tables                                                         */
/* ------------------------------------------------------------------------ */

/* Radon's 7-point rule, exact for polynomials of degree <= 5 on a triangle
 * (Stroud's T2:5-1).  Barycentric nodes, weights summing to one. */
void or_radon7(double lam[21], double w[7])
{
    double s = sqrt(15.0);
    double a1 = (6.0 - s) / 21.0, b1 = (9.0 + 2.0 * s) / 21.0;
    double a2 = (6.0 + s) / 21.0, b2 = (9.0 - 2.0 * s) / 21.0;
    double w1 = (155.0 - s) / 1200.0, w2 = (155.0 + s) / 1200.0;
    double L[7][3] = {
        {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0},
        {a1, a1, b1}, {a1, b1, a1}, {b1, a1, a1},
        {a2, a2, b2}, {a2, b2, a2}, {b2, a2, a2}};
    double W[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
    for (int q = 0; q < 7; ++q) {
        for (int c = 0; c < 3; ++c) lam[3 * q + c] = L[q][c];
        w[q] = W[q];
    }
}

/* n-point Gauss-Legendre rule on [0,1]: roots of P_n by Newton's method on the
 * three-term recurrence (k+1) P_{k+1} = (2k+1) t P_k - k P_{k-1}, weights
 * 2 / ((1 - t^2) P_n'(t)^2), then mapped from [-1,1] to [0,1]. */
void or_gauss_legendre01(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double t = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = t;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
        }
        double wt = 2.0 / ((1.0 - t * t) * dp * dp);
        x[n - 1 - i] = 0.5 * (t + 1.0);
        w[n - 1 - i] = 0.5 * wt;
    }
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */

static void centroid(const double* a, const double* b, const double* c, double g[3])
{
    for (int k = 0; k < 3; ++k) g[k] = (a[k] + b[k] + c[k]) / 3.0;
}

static double dist2(const double* a, const double* b)
{
    double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
    return d0 * d0 + d1 * d1 + d2 * d2;
}

static double tri_diam2(const double* a, const double* b, const double* c)
{
    double e0 = dist2(a, b), e1 = dist2(b, c), e2 = dist2(c, a);
    double m = e0 > e1 ? e0 : e1;
    return m > e2 ? m : e2;
}

static double tri_area(const double* a, const double* b, const double* c)
{
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double n0 = u[1] * v[2] - u[2] * v[1];
    double n1 = u[2] * v[0] - u[0] * v[2];
    double n2 = u[0] * v[1] - u[1] * v[0];
    return 0.5 * sqrt(n0 * n0 + n1 * n1 + n2 * n2);
}

/* Collocation points: the centroid of every triangle (row-major M x 3). */
void or_centroids(const double* V, const int32_t* T, int64_t M, double* C)
{
    for (int64_t i = 0; i < M; ++i)
        centroid(V + 3 * T[3 * i], V + 3 * T[3 * i + 1], V + 3 * T[3 * i + 2], C + 3 * i);
}

/* ------------------------------------------------------------------------ */
/* Integrands                                                                */
/* ------------------------------------------------------------------------ */

/* The seven scalar kernels of Eq. (Vh) at one source point y, without the
 * 1/(4 pi) factor: [1/r, d0 d0/r^3, d0 d1/r^3, d0 d2/r^3, d1 d1/r^3,
 * d1 d2/r^3, d2 d2/r^3] with d = x - y. */
static void scalar_kernels_at(const double* x, const double* y, double f[7])
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double r = sqrt(r2);
    double ir = 1.0 / r;
    double ir3 = ir / r2;
    f[0] = ir;
    f[1] = d[0] * d[0] * ir3;
    f[2] = d[0] * d[1] * ir3;
    f[3] = d[0] * d[2] * ir3;
    f[4] = d[1] * d[1] * ir3;
    f[5] = d[1] * d[2] * ir3;
    f[6] = d[2] * d[2] * ir3;
}

/* Kelvin's solution tensor S_K(d), Section 4.1, row-major 3 x 3. */
static void kelvin_at(const double* x, const double* y, double E, double nu, double S[9])
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double r = sqrt(r2);
    double pref = (1.0 / (8.0 * OR_PI)) * (1.0 / E) * ((1.0 + nu) / (1.0 - nu));
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double delta = (a == b) ? 1.0 : 0.0;
            S[3 * a + b] = pref * ((3.0 - 4.0 * nu) * delta / r + d[a] * d[b] / (r2 * r));
        }
}

/* A generic "value at a source point" so that the same quadrature serves the
 * seven scalar kernels and the Kelvin tensor. */
typedef struct {
    int nval;     /* 7 scalar kernels, 9 tensor entries, or 3 hat-weighted double-layer values */
    double E, nu; /* used by the tensor */
    /* the double layer: the triangle tau (vertices p[0..2]) whose hat
     * functions weight the kernel, its unit normal and (p1-p0)x(p2-p0).n */
    const double* p[3];
    double n[3], twice_area;
} integrand;

/* The double-layer kernel of Section 4.1's K (the Laplace part, K_Delta):
 * (x - y).n(y) / |x - y|^3 times the three barycentric coordinates of y in
 * tau (the hat functions psi_j of tau's vertices), without 1/(4 pi). */
static void double_layer_at(const integrand* g, const double* x, const double* y, double f[3])
{
    double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double r = sqrt(r2);
    double k = (d[0] * g->n[0] + d[1] * g->n[1] + d[2] * g->n[2]) / (r2 * r);
    for (int a = 0; a < 3; ++a) {
        const double* q1 = g->p[(a + 1) % 3];
        const double* q2 = g->p[(a + 2) % 3];
        double u[3] = {q1[0] - y[0], q1[1] - y[1], q1[2] - y[2]};
        double v[3] = {q2[0] - y[0], q2[1] - y[1], q2[2] - y[2]};
        double c0 = u[1] * v[2] - u[2] * v[1], c1 = u[2] * v[0] - u[0] * v[2], c2 = u[0] * v[1] - u[1] * v[0];
        double lam = (c0 * g->n[0] + c1 * g->n[1] + c2 * g->n[2]) / g->twice_area;
        f[a] = k * lam;
    }
}

static void eval_at(const integrand* g, const double* x, const double* y, double* f)
{
    if (g->nval == 7)
        scalar_kernels_at(x, y, f);
    else if (g->nval == 3)
        double_layer_at(g, x, y, f);
    else
        kelvin_at(x, y, g->E, g->nu, f);
}

/* 7-point rule on one (sub-)triangle: acc += area * sum_q w_q f(y_q). */
static void rule7(const integrand* g, const double* x, const double* a, const double* b,
                  const double* c, double* acc)
{
    double lam[21], w[7], f[9], s[9] = {0};
    or_radon7(lam, w);
    for (int q = 0; q < 7; ++q) {
        double y[3];
        for (int k = 0; k < 3; ++k)
            y[k] = lam[3 * q] * a[k] + lam[3 * q + 1] * b[k] + lam[3 * q + 2] * c[k];
        eval_at(g, x, y, f);
        for (int v = 0; v < g->nval; ++v) s[v] += w[q] * f[v];
    }
    double area = tri_area(a, b, c);
    for (int v = 0; v < g->nval; ++v) acc[v] += area * s[v];
}

/* Adaptive rule for x outside the triangle (a, b, c): subdivide into the four
 * midpoint triangles (corner a, corner b, corner c, middle) while the
 * centroid distance is below rho * diameter and depth < 8. */
static void adaptive(const integrand* g, const double* x, const double* a, const double* b,
                     const double* c, int depth, double* acc)
{
    double gc[3];
    centroid(a, b, c, gc);
    if (depth < OR_MAXDEPTH && dist2(x, gc) < OR_RHO2 * tri_diam2(a, b, c)) {
        double ab[3], bc[3], ca[3];
        for (int k = 0; k < 3; ++k) {
            ab[k] = (a[k] + b[k]) * 0.5;
            bc[k] = (b[k] + c[k]) * 0.5;
            ca[k] = (c[k] + a[k]) * 0.5;
        }
        adaptive(g, x, a, ab, ca, depth + 1, acc);
        adaptive(g, x, ab, b, bc, depth + 1, acc);
        adaptive(g, x, ca, bc, c, depth + 1, acc);
        adaptive(g, x, ab, bc, ca, depth + 1, acc);
        return;
    }
    rule7(g, x, a, b, c, acc);
}

/* Self pair: x is the centroid of (p0, p1, p2).  For each edge (pa, pb) the
 * sub-triangle (x, pa, pb) is parametrised y = x + u (a + v b), a = pa - x,
 * b = pb - pa, with surface element u |a x b| du dv.  Since x - y = -u e(v),
 * e = a + v b, every kernel here is homogeneous of degree -1 in x - y, so the
 * u-integral is exactly one and only int_0^1 |a x b| k(e(v)) dv remains. */
static void self_term(const integrand* g, const double* x, const double* p0, const double* p1,
                      const double* p2, int nd, double* acc)
{
    double vq[64], wq[64];
    if (nd < 1 || nd > 64) {
        /* outside the node tables: no value rather than an overrun */
        for (int v = 0; v < g->nval; ++v) acc[v] = NAN;
        return;
    }
    or_gauss_legendre01(nd, vq, wq);
    const double* P[3] = {p0, p1, p2};
    double zero[3] = {0.0, 0.0, 0.0};
    for (int e = 0; e < 3; ++e) {
        const double* pa = P[e];
        const double* pb = P[(e + 1) % 3];
        double a[3] = {pa[0] - x[0], pa[1] - x[1], pa[2] - x[2]};
        double b[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
        double n0 = a[1] * b[2] - a[2] * b[1];
        double n1 = a[2] * b[0] - a[0] * b[2];
        double n2 = a[0] * b[1] - a[1] * b[0];
        double cr = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
        double f[9];
        for (int q = 0; q < nd; ++q) {
            /* evaluate the kernel at "x - y = -e": pass x = 0 and y = -e,
             * i.e. d = e (the kernels are even in d) */
            double y[3];
            for (int k = 0; k < 3; ++k) y[k] = -(a[k] + vq[q] * b[k]);
            eval_at(g, zero, y, f);
            for (int v = 0; v < g->nval; ++v) acc[v] += wq[q] * cr * f[v];
        }
    }
}

static void pair_integral(const integrand* g, const double* x, const double* V,
                          const int32_t* tj, int self, int nd, double* out)
{
    const double* p0 = V + 3 * tj[0];
    const double* p1 = V + 3 * tj[1];
    const double* p2 = V + 3 * tj[2];
    for (int v = 0; v < g->nval; ++v) out[v] = 0.0;
    if (self)
        self_term(g, x, p0, p1, p2, nd, out);
    else
        adaptive(g, x, p0, p1, p2, 0, out);
}

/* The seven scalar kernels of Eq. (Vh) (collocation form, Section 4.2 with the
 * outer integral replaced by evaluation at x):
 *   out = (1/(4 pi)) int_{tau_j} [1/r, (x-y)_k (x-y)_l / r^3] ds_y.
 * self != 0 means x is the centroid of tau_j. */
void or_scalar_entry(const double* x, const double* V, const int32_t* tj, int self, int nd,
                     double out[7])
{
    integrand g = {7, 0.0, 0.0};
    pair_integral(&g, x, V, tj, self, nd, out);
    for (int v = 0; v < 7; ++v) out[v] *= 1.0 / (4.0 * OR_PI);
}

/* The 3 x 3 block int_{tau_j} S_K(x - y) ds_y computed from Kelvin's tensor
 * directly (Section 4.1), row-major. */
void or_kelvin_entry(const double* x, const double* V, const int32_t* tj, int self, int nd,
                     double E, double nu, double out[9])
{
    integrand g = {9, E, nu};
    pair_integral(&g, x, V, tj, self, nd, out);
}

/* Dense scalar-kernel matrices for rows `rows` (nr of them) and all M columns:
 * out[(v * nr + r) * M + j], v = 0..6. */
void or_scalar_rows(const double* V, const int32_t* T, int64_t M, const int64_t* rows,
                    int64_t nr, double* out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nr; ++r) {
        int64_t i = rows[r];
        double x[3], e[7];
        centroid(V + 3 * T[3 * i], V + 3 * T[3 * i + 1], V + 3 * T[3 * i + 2], x);
        for (int64_t j = 0; j < M; ++j) {
            or_scalar_entry(x, V, T + 3 * j, i == j, OR_ND, e);
            for (int v = 0; v < 7; ++v) out[(v * nr + r) * M + j] = e[v];
        }
    }
}

/* Exact (quadrature-contract) rows of the Kelvin product: for each sampled
 * triangle i and component a, y[3 r + a] = sum_j sum_b K_ab(i, j) x[3 j + b]. */
void or_kelvin_rows_matvec(const double* V, const int32_t* T, int64_t M, double E, double nu,
                           const int64_t* rows, int64_t nr, const double* x, int64_t nrhs,
                           double* y)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nr; ++r) {
        int64_t i = rows[r];
        double c[3], K[9];
        centroid(V + 3 * T[3 * i], V + 3 * T[3 * i + 1], V + 3 * T[3 * i + 2], c);
        for (int64_t q = 0; q < nrhs; ++q)
            for (int a = 0; a < 3; ++a) y[q * 3 * nr + 3 * r + a] = 0.0;
        for (int64_t j = 0; j < M; ++j) {
            or_kelvin_entry(c, V, T + 3 * j, i == j, OR_ND, E, nu, K);
            for (int64_t q = 0; q < nrhs; ++q) {
                const double* xq = x + q * 3 * M;
                for (int a = 0; a < 3; ++a) {
                    double s = 0.0;
                    for (int b = 0; b < 3; ++b) s += K[3 * a + b] * xq[3 * j + b];
                    y[q * 3 * nr + 3 * r + a] += s;
                }
            }
        }
    }
}

/* The evaluation operator of Section 5, Eq. (vector_eq) applied by its definition: for each
 * point x_r and component a, y[3 r + a] = sum_j sum_b int_{tau_j} S_ab(x_r - y)
 * ds_y x[3 j + b], Kelvin's tensor integrated directly (Section 4.1) with the
 * same quadrature as the collocation entries (x_r is never a centroid of its
 * own triangle: no self pair).  x is (nrhs, 3M), y (nrhs, 3 np). */
void or_kelvin_points_matvec(const double* V, const int32_t* T, int64_t M, double E, double nu,
                             const double* P, int64_t np, const double* x, int64_t nrhs, double* y)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < np; ++r) {
        double K[9];
        for (int64_t q = 0; q < nrhs; ++q)
            for (int a = 0; a < 3; ++a) y[q * 3 * np + 3 * r + a] = 0.0;
        for (int64_t j = 0; j < M; ++j) {
            or_kelvin_entry(P + 3 * r, V, T + 3 * j, 0, OR_ND, E, nu, K);
            for (int64_t q = 0; q < nrhs; ++q) {
                const double* xq = x + q * 3 * M;
                for (int a = 0; a < 3; ++a) {
                    double s = 0.0;
                    for (int b = 0; b < 3; ++b) s += K[3 * a + b] * xq[3 * j + b];
                    y[q * 3 * np + 3 * r + a] += s;
                }
            }
        }
    }
}

/* The seven scalar kernels at points P (np of them) against all M triangles:
 * out[(v * np + r) * M + j]. */
void or_scalar_points(const double* V, const int32_t* T, int64_t M, const double* P, int64_t np,
                      double* out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < np; ++r) {
        double e[7];
        for (int64_t j = 0; j < M; ++j) {
            or_scalar_entry(P + 3 * r, V, T + 3 * j, 0, OR_ND, e);
            for (int v = 0; v < 7; ++v) out[(v * np + r) * M + j] = e[v];
        }
    }
}

/* The double-layer block of Eq. (Kh), collocation at x (reading: the outer
 * integral over tau_i dropped, as for V_h):
 *   out[a] = (1/(4 pi)) int_{tau_j} (x - y).n_j / |x - y|^3 psi_a(y) ds_y
 * for the three vertices a of tau_j (psi_a the hat function of vertex a),
 * n_j the unit normal of tau_j from its vertex order.  self != 0 means x lies
 * in tau_j (its centroid): (x - y).n_j = 0 on the flat triangle, so the
 * values are exactly 0. */
void or_dl_entry(const double* x, const double* V, const int32_t* tj, int self, double out[3])
{
    for (int a = 0; a < 3; ++a) out[a] = 0.0;
    if (self) return;
    const double* p0 = V + 3 * tj[0];
    const double* p1 = V + 3 * tj[1];
    const double* p2 = V + 3 * tj[2];
    integrand g;
    memset(&g, 0, sizeof g);
    g.nval = 3;
    g.p[0] = p0;
    g.p[1] = p1;
    g.p[2] = p2;
    double e1[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
    double e2[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
    double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    for (int k = 0; k < 3; ++k) g.n[k] = c[k] / len;
    g.twice_area = len;
    adaptive(&g, x, p0, p1, p2, 0, out);
    for (int a = 0; a < 3; ++a) out[a] *= 1.0 / (4.0 * OR_PI);
}

/* Dense K_Delta of Eq. (Kh) at the collocation points: M x nv row-major,
 * out[i * nv + p] = sum over the triangles tau_j holding vertex p of the
 * entry of or_dl_entry(c_i, tau_j) for that vertex. */
void or_dl_dense(const double* V, int64_t nv, const int32_t* T, int64_t M, double* out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < M; ++i) {
        double x[3], e[3];
        centroid(V + 3 * T[3 * i], V + 3 * T[3 * i + 1], V + 3 * T[3 * i + 2], x);
        double* row = out + i * nv;
        for (int64_t p = 0; p < nv; ++p) row[p] = 0.0;
        for (int64_t j = 0; j < M; ++j) {
            or_dl_entry(x, V, T + 3 * j, i == j, e);
            for (int a = 0; a < 3; ++a) row[T[3 * j + a]] += e[a];
        }
    }
}

/* Dense Kelvin matrix, 3M x 3M row-major, dof 3 i + a. */
void or_kelvin_dense(const double* V, const int32_t* T, int64_t M, double E, double nu,
                     double* A)
{
    int64_t n = 3 * M;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < M; ++i) {
        double c[3], K[9];
        centroid(V + 3 * T[3 * i], V + 3 * T[3 * i + 1], V + 3 * T[3 * i + 2], c);
        for (int64_t j = 0; j < M; ++j) {
            or_kelvin_entry(c, V, T + 3 * j, i == j, OR_ND, E, nu, K);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) A[(3 * i + a) * n + 3 * j + b] = K[3 * a + b];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Cluster tree (Section 2.1)                                                */
/* ------------------------------------------------------------------------ */
/* Reading of the construction the paper defers to the literature: split a
 * cluster along the longest axis of the bounding box of its collocation
 * points (ties: lowest axis), at the median of a stable sort by
 * (coordinate, original index); the first son gets floor(n/2) indices.  A
 * cluster with at most `leaf` indices is a leaf.  Nodes are numbered in
 * depth-first pre-order; the leaves in that order define the cluster order. */

typedef struct {
    int64_t lo, hi;   /* [lo, hi) in cluster order */
    int64_t son[2];   /* -1 for a leaf */
    int32_t level;
    double bmin[3], bmax[3]; /* box of all triangle vertices of the cluster (of
                                the points, in a tree of points) */
} or_node;

typedef struct {
    const double* key;
    int64_t idx;
} sort_item;

static int cmp_item(const void* pa, const void* pb)
{
    const sort_item* a = (const sort_item*)pa;
    const sort_item* b = (const sort_item*)pb;
    if (*a->key < *b->key) return -1;
    if (*a->key > *b->key) return 1;
    return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

typedef struct {
    const double* V;
    const int32_t* T;
    const double* C;
    int64_t leaf;
    int64_t* perm;
    or_node* nodes;
    int64_t nn;
    sort_item* tmp;
    const double* B;  /* without T: a box per item (min xyz, max xyz), else the item is a point */
} tree_ctx;

static int64_t build_node(tree_ctx* tc, int64_t lo, int64_t hi, int32_t level)
{
    int64_t id = tc->nn++;
    or_node* nd = &tc->nodes[id];
    nd->lo = lo;
    nd->hi = hi;
    nd->level = level;
    nd->son[0] = nd->son[1] = -1;
    for (int k = 0; k < 3; ++k) {
        nd->bmin[k] = INFINITY;
        nd->bmax[k] = -INFINITY;
    }
    for (int64_t p = lo; p < hi; ++p) {
        if (!tc->T) {
            /* a tree of points: the box of the points themselves; with item
             * boxes (the supports of hat functions) their union */
            for (int k = 0; k < 3; ++k) {
                double lo = tc->B ? tc->B[6 * tc->perm[p] + k] : tc->C[3 * tc->perm[p] + k];
                double hi = tc->B ? tc->B[6 * tc->perm[p] + 3 + k] : tc->C[3 * tc->perm[p] + k];
                if (lo < nd->bmin[k]) nd->bmin[k] = lo;
                if (hi > nd->bmax[k]) nd->bmax[k] = hi;
            }
            continue;
        }
        const int32_t* t = tc->T + 3 * tc->perm[p];
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 3; ++k) {
                double v = tc->V[3 * t[c] + k];
                if (v < nd->bmin[k]) nd->bmin[k] = v;
                if (v > nd->bmax[k]) nd->bmax[k] = v;
            }
    }
    if (hi - lo <= tc->leaf) return id;
    double cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t p = lo; p < hi; ++p)
        for (int k = 0; k < 3; ++k) {
            double v = tc->C[3 * tc->perm[p] + k];
            if (v < cmin[k]) cmin[k] = v;
            if (v > cmax[k]) cmax[k] = v;
        }
    int ax = 0;
    double best = cmax[0] - cmin[0];
    for (int k = 1; k < 3; ++k)
        if (cmax[k] - cmin[k] > best) {
            best = cmax[k] - cmin[k];
            ax = k;
        }
    for (int64_t p = lo; p < hi; ++p) {
        tc->tmp[p - lo].idx = tc->perm[p];
        tc->tmp[p - lo].key = tc->C + 3 * tc->perm[p] + ax;
    }
    qsort(tc->tmp, (size_t)(hi - lo), sizeof(sort_item), cmp_item);
    for (int64_t p = lo; p < hi; ++p) tc->perm[p] = tc->tmp[p - lo].idx;
    int64_t mid = lo + (hi - lo) / 2;
    int64_t s0 = build_node(tc, lo, mid, level + 1);
    int64_t s1 = build_node(tc, mid, hi, level + 1);
    tc->nodes[id].son[0] = s0;
    tc->nodes[id].son[1] = s1;
    return id;
}

/* ------------------------------------------------------------------------ */
/* Block partition (Section 2.1, Eq. (adm))                                  */
/* ------------------------------------------------------------------------ */
/* Admissible iff min(diam B_t, diam B_s) < eta dist(B_t, B_s) for the vertex
 * boxes (a superset of X_t, X_s, so the test stays sufficient); compared in
 * squares.  Otherwise split both clusters if neither is a leaf, only the
 * non-leaf one if one is a leaf, and emit a near block if both are leaves.
 * Rows and columns may come from different trees (the evaluation operator of
 * Section 5, Eq. (vector_eq): a tree of points times the triangle tree). */

typedef struct {
    int64_t t, s;
} or_block;

typedef struct {
    or_block* adm;
    int64_t nadm, capadm;
    or_block* near;
    int64_t nnear, capnear;
} block_lists;

static void push_block(or_block** arr, int64_t* n, int64_t* cap, int64_t t, int64_t s)
{
    if (*n == *cap) {
        *cap = *cap ? 2 * *cap : 1024;
        *arr = (or_block*)realloc(*arr, (size_t)(*cap) * sizeof(or_block));
    }
    (*arr)[*n].t = t;
    (*arr)[*n].s = s;
    ++*n;
}

static double box_diam2(const or_node* a)
{
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double e = a->bmax[k] - a->bmin[k];
        s += e * e;
    }
    return s;
}

static double box_dist2(const or_node* a, const or_node* b)
{
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double g1 = a->bmin[k] - b->bmax[k];
        double g2 = b->bmin[k] - a->bmax[k];
        double g = g1 > g2 ? g1 : g2;
        if (g < 0.0) g = 0.0;
        s += g * g;
    }
    return s;
}

static void partition(const or_node* rnodes, const or_node* nodes, int64_t t, int64_t s, double eta,
                      block_lists* bl)
{
    const or_node* a = &rnodes[t];
    const or_node* b = &nodes[s];
    double da = box_diam2(a), db = box_diam2(b);
    double dmin = da < db ? da : db;
    if (dmin < (eta * eta) * box_dist2(a, b)) {
        push_block(&bl->adm, &bl->nadm, &bl->capadm, t, s);
        return;
    }
    int tl = a->son[0] < 0, sl = b->son[0] < 0;
    if (!tl && !sl) {
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) partition(rnodes, nodes, a->son[p], b->son[q], eta, bl);
    } else if (!tl) {
        for (int p = 0; p < 2; ++p) partition(rnodes, nodes, a->son[p], s, eta, bl);
    } else if (!sl) {
        for (int q = 0; q < 2; ++q) partition(rnodes, nodes, t, b->son[q], eta, bl);
    } else {
        push_block(&bl->near, &bl->nnear, &bl->capnear, t, s);
    }
}

/* ------------------------------------------------------------------------ */
/* ACA, Algorithm 1                                                          */
/* ------------------------------------------------------------------------ */
/* Readings (the paper leaves them open):
 *   first row: the first index of t; "does not vanish": max|v~| > delta max|raw row|
 *   (delta = 1e-14); after a vanishing row the next row is the argmax of the last
 *   u over rows not in Z, or the smallest row not in Z if there is no usable u;
 *   argmax ties: the smallest index whose modulus is within a relative 1e-10 of
 *   the maximum; stop test on the newest cross against ||S_k||_F (which includes
 *   it), with factor eps (1 - eta_stop) / (1 + eps); ||S_k||_F^2 by the recursive
 *   update ||S_{k-1}||^2 + 2 sum_{l<k} (u_k.u_l)(v_l.v_k) + |u_k|^2 |v_k|^2;
 *   also stop when Z = t, when k = min(m, n) or at the rank cap kmax. */

#define OR_ACA_DELTA 1e-14
#define OR_ACA_TIE 1e-10

typedef void (*or_row_fn)(void* ctx, int64_t i, double* out);  /* A[i, s] (n values) */
typedef void (*or_col_fn)(void* ctx, int64_t j, double* out);  /* A[t, j] (m values) */

typedef struct {
    int32_t rank;
    int32_t steps;      /* rows visited (accepted + vanished) */
    int32_t flags;      /* 1: rank cap reached, 2: Z exhausted, 4: k = min(m,n),
                           32 (set by the H-matrix build): kernel identically zero */
} or_aca_info;

/* smallest index among the entries (with mask[i] == 0 if mask) whose modulus is
 * within the tie tolerance of the maximum modulus; -1 if none / maximum is 0 */
static int64_t pick_pivot(const double* v, int64_t n, const unsigned char* mask, double* maxout)
{
    double mx = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (mask && mask[i]) continue;
        double a = fabs(v[i]);
        if (a > mx) mx = a;
    }
    if (maxout) *maxout = mx;
    if (!(mx > 0.0)) return -1;
    double thr = mx * (1.0 - OR_ACA_TIE);
    for (int64_t i = 0; i < n; ++i) {
        if (mask && mask[i]) continue;
        if (fabs(v[i]) >= thr) return i;
    }
    return -1;
}

/* U is m x kmax column-major (column l at U + l*m), V is n x kmax. Returns rank. */
int32_t or_aca(int64_t m, int64_t n, or_row_fn rowf, or_col_fn colf, void* ctx, double eps,
               double eta_stop, int32_t kmax, double* U, double* Vf, int64_t* piv_i,
               int64_t* piv_j, or_aca_info* info)
{
    unsigned char* Z = (unsigned char*)calloc((size_t)m, 1);
    double* raw = (double*)malloc((size_t)(n > m ? n : m) * sizeof(double));
    int64_t nz = 0;
    int32_t k = 0, steps = 0, flags = 0;
    double S2 = 0.0;
    double fac = eps * (1.0 - eta_stop) / (1.0 + eps);
    int64_t kcap = kmax;
    if (kcap > m) kcap = m;
    if (kcap > n) kcap = n;
    int64_t i = 0;
    while (1) {
        if (k >= kmax) {
            flags |= 1;
            break;
        }
        /* residual row  v~ = A[i, s] - sum_{l<k} (u_l)_i v_l */
        double* vt = Vf + (int64_t)k * n;
        rowf(ctx, i, raw);
        double mraw = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double s = raw[j];
            for (int32_t l = 0; l < k; ++l) s -= U[(int64_t)l * m + i] * Vf[(int64_t)l * n + j];
            vt[j] = s;
            if (fabs(raw[j]) > mraw) mraw = fabs(raw[j]);
        }
        ++steps;
        Z[i] = 1;
        ++nz;
        double mres = 0.0;
        int64_t jk = pick_pivot(vt, n, NULL, &mres);
        if (jk < 0 || mres <= OR_ACA_DELTA * mraw) {
            /* vanishing row: choose another row and try again */
            if (nz == m) {
                flags |= 2;
                break;
            }
            int64_t nxt = -1;
            if (k > 0) nxt = pick_pivot(U + (int64_t)(k - 1) * m, m, Z, NULL);
            if (nxt < 0)
                for (int64_t r = 0; r < m; ++r)
                    if (!Z[r]) {
                        nxt = r;
                        break;
                    }
            i = nxt;
            continue;
        }
        /* v_k = v~ / v~_{jk} */
        double inv = 1.0 / vt[jk];
        for (int64_t j = 0; j < n; ++j) vt[j] = vt[j] * inv;
        /* u_k = A[t, jk] - sum_{l<k} (v_l)_{jk} u_l */
        double* uk = U + (int64_t)k * m;
        colf(ctx, jk, raw);
        for (int64_t r = 0; r < m; ++r) {
            double s = raw[r];
            for (int32_t l = 0; l < k; ++l) s -= Vf[(int64_t)l * n + jk] * U[(int64_t)l * m + r];
            uk[r] = s;
        }
        if (piv_i) piv_i[k] = i;
        if (piv_j) piv_j[k] = jk;
        /* recursive Frobenius norm of S_k */
        double uu = 0.0, vv = 0.0;
        for (int64_t r = 0; r < m; ++r) uu += uk[r] * uk[r];
        for (int64_t j = 0; j < n; ++j) vv += vt[j] * vt[j];
        double cross = 0.0;
        for (int32_t l = 0; l < k; ++l) {
            double a = 0.0, b = 0.0;
            for (int64_t r = 0; r < m; ++r) a += uk[r] * U[(int64_t)l * m + r];
            for (int64_t j = 0; j < n; ++j) b += Vf[(int64_t)l * n + j] * vt[j];
            cross += a * b;
        }
        S2 = S2 + 2.0 * cross + uu * vv;
        ++k;
        if (sqrt(uu * vv) <= fac * sqrt(S2 > 0.0 ? S2 : 0.0)) break;
        if (nz == m) {
            flags |= 2;
            break;
        }
        if (k >= kcap) {
            flags |= 4;
            break;
        }
        i = pick_pivot(uk, m, Z, NULL);
        if (i < 0)
            for (int64_t r = 0; r < m; ++r)
                if (!Z[r]) {
                    i = r;
                    break;
                }
    }
    free(Z);
    free(raw);
    if (info) {
        info->rank = k;
        info->steps = steps;
        info->flags = flags;
    }
    return k;
}

/* ACA on an explicit dense block A (m x n, row-major): used to pin Algorithm 1
 * on synthetic matrices. */
typedef struct {
    const double* A;
    int64_t m, n;
} dense_ctx;

static void dense_row(void* c, int64_t i, double* out)
{
    dense_ctx* d = (dense_ctx*)c;
    memcpy(out, d->A + i * d->n, (size_t)d->n * sizeof(double));
}

static void dense_col(void* c, int64_t j, double* out)
{
    dense_ctx* d = (dense_ctx*)c;
    for (int64_t i = 0; i < d->m; ++i) out[i] = d->A[i * d->n + j];
}

int32_t or_aca_dense(const double* A, int64_t m, int64_t n, double eps, double eta_stop,
                     int32_t kmax, double* U, double* Vf, int64_t* piv_i, int64_t* piv_j,
                     int32_t* steps, int32_t* flags)
{
    dense_ctx d = {A, m, n};
    or_aca_info info;
    int32_t k = or_aca(m, n, dense_row, dense_col, &d, eps, eta_stop, kmax, U, Vf, piv_i, piv_j,
                       &info);
    if (steps) *steps = info.steps;
    if (flags) *flags = info.flags;
    return k;
}

/* ------------------------------------------------------------------------ */
/* Oracle H-matrix                                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t M, nv;
    double* V;       /* copy of the mesh */
    int32_t* T;
    double* C;       /* collocation points, original order */
    int64_t* perm;   /* cluster position -> original triangle */
    or_node* nodes;
    int64_t nnodes;
    /* rows: the collocation points themselves (square), or the points x_i of
     * the evaluation operator ~V_h (Section 5, Eq. (vector_eq)) with their own tree */
    int square;
    int64_t Mr;
    double* X;       /* row points, original order (== C when square) */
    int64_t* rperm;  /* row cluster position -> original row */
    or_node* rnodes;
    int64_t nrnodes;
    block_lists bl;
    double eps, eta, eta_stop;
    int32_t kmax;
    /* per admissible block and kernel: rank and factors (original-order rows
     * are reached through perm) */
    int32_t* rank;       /* nadm * 7 */
    double** Uf;         /* nadm * 7 pointers, |t| x rank column-major */
    double** Vf;         /* nadm * 7 pointers, |s| x rank column-major */
    int32_t* aca_flags;  /* nadm * 7 */
    /* near blocks: |t| x |s| x 9 Kelvin blocks are material dependent, so
     * store the seven scalar kernels: 7 x |t| x |s| */
    double** Nf;         /* nnear pointers */
    unsigned char* adm_done;
    unsigned char* near_done;
} or_hmat;

typedef struct {
    const or_hmat* h;
    int64_t t0, s0, m, n;
    int kern;
    double* tmp7;
} kernel_ctx;

static void kernel_entry(const or_hmat* h, int64_t pi, int64_t pj, double e[7])
{
    int64_t i = h->rperm[pi], j = h->perm[pj];
    or_scalar_entry(h->X + 3 * i, h->V, h->T + 3 * j, h->square && i == j, OR_ND, e);
}

static void kernel_row(void* c, int64_t i, double* out)
{
    kernel_ctx* k = (kernel_ctx*)c;
    double e[7];
    for (int64_t j = 0; j < k->n; ++j) {
        kernel_entry(k->h, k->t0 + i, k->s0 + j, e);
        out[j] = e[k->kern];
    }
}

static void kernel_col(void* c, int64_t j, double* out)
{
    kernel_ctx* k = (kernel_ctx*)c;
    double e[7];
    for (int64_t i = 0; i < k->m; ++i) {
        kernel_entry(k->h, k->t0 + i, k->s0 + j, e);
        out[i] = e[k->kern];
    }
}

/* the triangle tree (columns); rows and partition are set by the callers */
static or_hmat* hmat_columns(const double* V, int64_t nv, const int32_t* T, int64_t M, int64_t leaf)
{
    or_hmat* h = (or_hmat*)calloc(1, sizeof(or_hmat));
    h->M = M;
    h->nv = nv;
    h->V = (double*)malloc((size_t)nv * 3 * sizeof(double));
    memcpy(h->V, V, (size_t)nv * 3 * sizeof(double));
    h->T = (int32_t*)malloc((size_t)M * 3 * sizeof(int32_t));
    memcpy(h->T, T, (size_t)M * 3 * sizeof(int32_t));
    h->C = (double*)malloc((size_t)M * 3 * sizeof(double));
    or_centroids(h->V, h->T, M, h->C);
    h->perm = (int64_t*)malloc((size_t)M * sizeof(int64_t));
    for (int64_t i = 0; i < M; ++i) h->perm[i] = i;
    h->nodes = (or_node*)malloc((size_t)(2 * M + 1) * sizeof(or_node));
    tree_ctx tc = {h->V, h->T, h->C, leaf, h->perm, h->nodes, 0,
                   (sort_item*)malloc((size_t)M * sizeof(sort_item))};
    build_node(&tc, 0, M, 0);
    free(tc.tmp);
    h->nnodes = tc.nn;
    return h;
}

/* the block storage once the partition is known */
static void hmat_blocks(or_hmat* h, double eta, double eps, double eta_stop, int32_t kmax)
{
    partition(h->rnodes, h->nodes, 0, 0, eta, &h->bl);
    h->eps = eps;
    h->eta = eta;
    h->eta_stop = eta_stop;
    h->kmax = kmax;
    int64_t na = h->bl.nadm, nn = h->bl.nnear;
    h->rank = (int32_t*)calloc((size_t)(na * 7 + 1), sizeof(int32_t));
    h->aca_flags = (int32_t*)calloc((size_t)(na * 7 + 1), sizeof(int32_t));
    h->Uf = (double**)calloc((size_t)(na * 7 + 1), sizeof(double*));
    h->Vf = (double**)calloc((size_t)(na * 7 + 1), sizeof(double*));
    h->Nf = (double**)calloc((size_t)(nn + 1), sizeof(double*));
    h->adm_done = (unsigned char*)calloc((size_t)(na + 1), 1);
    h->near_done = (unsigned char*)calloc((size_t)(nn + 1), 1);
}

void* or_hmat_create(const double* V, int64_t nv, const int32_t* T, int64_t M, int64_t leaf,
                     double eta, double eps, double eta_stop, int32_t kmax)
{
    or_hmat* h = hmat_columns(V, nv, T, M, leaf);
    h->square = 1;
    h->Mr = M;
    h->X = h->C;
    h->rperm = h->perm;
    h->rnodes = h->nodes;
    h->nrnodes = h->nnodes;
    hmat_blocks(h, eta, eps, eta_stop, kmax);
    return h;
}

/* The evaluation operator ~V_h of Section 5, Eq. (vector_eq) (the displacement at points
 * x_1 .. x_np of the domain): rows are the points, clustered by the same
 * rule as the triangles with the boxes of the points, columns the triangles;
 * the entries are the collocation entries with x_i in place of a centroid
 * (never a self pair). */
void* or_hmat_points_create(const double* V, int64_t nv, const int32_t* T, int64_t M, int64_t leaf,
                            const double* P, int64_t np, int64_t leaf_pts, double eta, double eps,
                            double eta_stop, int32_t kmax)
{
    or_hmat* h = hmat_columns(V, nv, T, M, leaf);
    h->square = 0;
    h->Mr = np;
    h->X = (double*)malloc((size_t)np * 3 * sizeof(double));
    memcpy(h->X, P, (size_t)np * 3 * sizeof(double));
    h->rperm = (int64_t*)malloc((size_t)np * sizeof(int64_t));
    for (int64_t i = 0; i < np; ++i) h->rperm[i] = i;
    h->rnodes = (or_node*)malloc((size_t)(2 * np + 1) * sizeof(or_node));
    tree_ctx tc = {NULL, NULL, h->X, leaf_pts, h->rperm, h->rnodes, 0,
                   (sort_item*)malloc((size_t)np * sizeof(sort_item))};
    build_node(&tc, 0, np, 0);
    free(tc.tmp);
    h->nrnodes = tc.nn;
    hmat_blocks(h, eta, eps, eta_stop, kmax);
    return h;
}

void or_hmat_free(void* hp)
{
    or_hmat* h = (or_hmat*)hp;
    if (!h) return;
    for (int64_t b = 0; b < h->bl.nadm * 7; ++b) {
        free(h->Uf[b]);
        free(h->Vf[b]);
    }
    for (int64_t b = 0; b < h->bl.nnear; ++b) free(h->Nf[b]);
    free(h->Uf);
    free(h->Vf);
    free(h->Nf);
    free(h->rank);
    free(h->aca_flags);
    free(h->adm_done);
    free(h->near_done);
    free(h->bl.adm);
    free(h->bl.near);
    if (!h->square) {
        free(h->X);
        free(h->rperm);
        free(h->rnodes);
    }
    free(h->nodes);
    free(h->perm);
    free(h->C);
    free(h->T);
    free(h->V);
    free(h);
}

void or_hmat_sizes(const void* hp, int64_t* out4)
{
    const or_hmat* h = (const or_hmat*)hp;
    out4[0] = h->nnodes;
    out4[1] = h->bl.nadm;
    out4[2] = h->bl.nnear;
    out4[3] = h->M;
}

/* rows: out2 = (row tree nodes, rows) */
void or_hmat_rsizes(const void* hp, int64_t* out2)
{
    const or_hmat* h = (const or_hmat*)hp;
    out2[0] = h->nrnodes;
    out2[1] = h->Mr;
}

static void export_tree(const or_node* nodes, int64_t nnodes, const int64_t* p, int64_t n, int64_t* perm,
                        int64_t* nodes5, double* boxes6)
{
    memcpy(perm, p, (size_t)n * sizeof(int64_t));
    for (int64_t q = 0; q < nnodes; ++q) {
        const or_node* nd = &nodes[q];
        nodes5[5 * q + 0] = nd->lo;
        nodes5[5 * q + 1] = nd->hi;
        nodes5[5 * q + 2] = nd->son[0];
        nodes5[5 * q + 3] = nd->son[1];
        nodes5[5 * q + 4] = nd->level;
        for (int k = 0; k < 3; ++k) {
            boxes6[6 * q + k] = nd->bmin[k];
            boxes6[6 * q + 3 + k] = nd->bmax[k];
        }
    }
}

/* the row tree (the point tree of an evaluation operator; the triangle tree
 * of a square one), as or_hmat_tree */
void or_hmat_rtree(const void* hp, int64_t* perm, int64_t* nodes5, double* boxes6)
{
    const or_hmat* h = (const or_hmat*)hp;
    export_tree(h->rnodes, h->nrnodes, h->rperm, h->Mr, perm, nodes5, boxes6);
}

/* perm[M]; nodes as int64 rows [lo, hi, son0, son1, level]; boxes as 6 doubles */
void or_hmat_tree(const void* hp, int64_t* perm, int64_t* nodes5, double* boxes6)
{
    const or_hmat* h = (const or_hmat*)hp;
    export_tree(h->nodes, h->nnodes, h->perm, h->M, perm, nodes5, boxes6);
}

/* ------------------------------------------------------------------------ */
/* The partition of the double layer's K_Delta (Eq. (Kh)): rows are the      */
/* triangles (collocation points), columns the vertices (hat functions)       */
/* ------------------------------------------------------------------------ */
/* The vertices are clustered by the triangles' rule (longest axis of the box
 * of the vertex coordinates, median of (coordinate, id), first son
 * floor(n/2), leaves of at most leaf_v); a cluster's box is the union of its
 * vertices' stars (the boxes of all triangles holding the vertex: the support
 * of its hat function), so that Eq. (adm) keeps every admissible block away
 * from the kernel's singularity. */
typedef struct {
    int64_t M, nv;
    int64_t* tperm;
    or_node* tnodes;
    int64_t ntn;
    int64_t* vperm;
    or_node* vnodes;
    int64_t nvn;
    block_lists bl;
} or_vpart;

void* or_vpart_create(const double* V, int64_t nv, const int32_t* T, int64_t M, int64_t leaf, int64_t leaf_v,
                      double eta)
{
    or_vpart* h = (or_vpart*)calloc(1, sizeof(or_vpart));
    h->M = M;
    h->nv = nv;
    double* C = (double*)malloc((size_t)M * 3 * sizeof(double));
    or_centroids(V, T, M, C);
    h->tperm = (int64_t*)malloc((size_t)M * sizeof(int64_t));
    for (int64_t i = 0; i < M; ++i) h->tperm[i] = i;
    h->tnodes = (or_node*)malloc((size_t)(2 * M + 1) * sizeof(or_node));
    tree_ctx tc = {V, T, C, leaf, h->tperm, h->tnodes, 0, (sort_item*)malloc((size_t)M * sizeof(sort_item)), NULL};
    build_node(&tc, 0, M, 0);
    free(tc.tmp);
    h->ntn = tc.nn;
    /* stars: the box of every triangle, merged into its three vertices */
    double* B = (double*)malloc((size_t)nv * 6 * sizeof(double));
    for (int64_t p = 0; p < nv; ++p)
        for (int k = 0; k < 3; ++k) {
            B[6 * p + k] = INFINITY;
            B[6 * p + 3 + k] = -INFINITY;
        }
    for (int64_t i = 0; i < M; ++i) {
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 3; ++k) {
                double v = V[3 * T[3 * i + c] + k];
                if (v < lo[k]) lo[k] = v;
                if (v > hi[k]) hi[k] = v;
            }
        for (int c = 0; c < 3; ++c) {
            int64_t p = T[3 * i + c];
            for (int k = 0; k < 3; ++k) {
                if (lo[k] < B[6 * p + k]) B[6 * p + k] = lo[k];
                if (hi[k] > B[6 * p + 3 + k]) B[6 * p + 3 + k] = hi[k];
            }
        }
    }
    h->vperm = (int64_t*)malloc((size_t)nv * sizeof(int64_t));
    for (int64_t p = 0; p < nv; ++p) h->vperm[p] = p;
    h->vnodes = (or_node*)malloc((size_t)(2 * nv + 1) * sizeof(or_node));
    tree_ctx tv = {NULL, NULL, V, leaf_v, h->vperm, h->vnodes, 0, (sort_item*)malloc((size_t)nv * sizeof(sort_item)), B};
    build_node(&tv, 0, nv, 0);
    free(tv.tmp);
    h->nvn = tv.nn;
    partition(h->tnodes, h->vnodes, 0, 0, eta, &h->bl);
    free(B);
    free(C);
    return h;
}

void or_vpart_sizes(const void* hp, int64_t* out4)
{
    const or_vpart* h = (const or_vpart*)hp;
    out4[0] = h->nvn;
    out4[1] = h->bl.nadm;
    out4[2] = h->bl.nnear;
    out4[3] = h->nv;
}

void or_vpart_tree(const void* hp, int64_t* perm, int64_t* nodes5, double* boxes6)
{
    const or_vpart* h = (const or_vpart*)hp;
    export_tree(h->vnodes, h->nvn, h->vperm, h->nv, perm, nodes5, boxes6);
}

void or_vpart_blocks(const void* hp, int64_t* adm, int64_t* nearb)
{
    const or_vpart* h = (const or_vpart*)hp;
    for (int64_t b = 0; b < h->bl.nadm; ++b) {
        adm[2 * b] = h->bl.adm[b].t;
        adm[2 * b + 1] = h->bl.adm[b].s;
    }
    for (int64_t b = 0; b < h->bl.nnear; ++b) {
        nearb[2 * b] = h->bl.near[b].t;
        nearb[2 * b + 1] = h->bl.near[b].s;
    }
}

void or_vpart_free(void* hp)
{
    or_vpart* h = (or_vpart*)hp;
    if (!h) return;
    free(h->bl.adm);
    free(h->bl.near);
    free(h->tperm);
    free(h->tnodes);
    free(h->vperm);
    free(h->vnodes);
    free(h);
}

/* block lists as node ids: adm[2*b], adm[2*b+1] = (t, s) */
void or_hmat_blocks(const void* hp, int64_t* adm, int64_t* nearb)
{
    const or_hmat* h = (const or_hmat*)hp;
    for (int64_t b = 0; b < h->bl.nadm; ++b) {
        adm[2 * b] = h->bl.adm[b].t;
        adm[2 * b + 1] = h->bl.adm[b].s;
    }
    for (int64_t b = 0; b < h->bl.nnear; ++b) {
        nearb[2 * b] = h->bl.near[b].t;
        nearb[2 * b + 1] = h->bl.near[b].s;
    }
}

/* Component pair (p, q) of the scalar kernels 1..6 (V_11, V_12, V_13, V_22, V_23, V_33). */
static const int kern_p[7] = {-1, 0, 0, 0, 1, 1, 2};
static const int kern_q[7] = {-1, 0, 1, 2, 1, 2, 2};

/* A kernel with factor (x - y)_a vanishes identically on a block whose
 * clusters' vertices all share the coordinate a (then every collocation point
 * and every source point has it too): its exact rank is 0, which is what
 * Algorithm 1 reaches in exact arithmetic once Z = t. */
static int kernel_vanishes(const or_node* t, const or_node* s, int kern)
{
    if (kern == 0) return 0;
    const int ax[2] = {kern_p[kern], kern_q[kern]};
    for (int e = 0; e < 2; ++e) {
        const int a = ax[e];
        if (t->bmin[a] == t->bmax[a] && s->bmin[a] == s->bmax[a] && t->bmin[a] == s->bmin[a]) return 1;
    }
    return 0;
}

static void assemble_adm(or_hmat* h, int64_t b)
{
    const or_node* t = &h->rnodes[h->bl.adm[b].t];
    const or_node* s = &h->nodes[h->bl.adm[b].s];
    int64_t m = t->hi - t->lo, n = s->hi - s->lo;
    for (int kern = 0; kern < 7; ++kern) {
        if (kernel_vanishes(t, s, kern)) {
            h->rank[b * 7 + kern] = 0;
            h->aca_flags[b * 7 + kern] = 32;
            h->Uf[b * 7 + kern] = (double*)malloc(sizeof(double));
            h->Vf[b * 7 + kern] = (double*)malloc(sizeof(double));
            continue;
        }
        int64_t kc = h->kmax;
        double* U = (double*)malloc((size_t)(m * kc) * sizeof(double));
        double* Vv = (double*)malloc((size_t)(n * kc) * sizeof(double));
        kernel_ctx kc_ = {h, t->lo, s->lo, m, n, kern, NULL};
        or_aca_info info;
        int32_t k = or_aca(m, n, kernel_row, kernel_col, &kc_, h->eps, h->eta_stop, h->kmax, U,
                           Vv, NULL, NULL, &info);
        h->rank[b * 7 + kern] = k;
        h->aca_flags[b * 7 + kern] = info.flags;
        h->Uf[b * 7 + kern] = (double*)realloc(U, (size_t)(m * (k ? k : 1)) * sizeof(double));
        h->Vf[b * 7 + kern] = (double*)realloc(Vv, (size_t)(n * (k ? k : 1)) * sizeof(double));
    }
    h->adm_done[b] = 1;
}

static void assemble_near(or_hmat* h, int64_t b)
{
    const or_node* t = &h->rnodes[h->bl.near[b].t];
    const or_node* s = &h->nodes[h->bl.near[b].s];
    int64_t m = t->hi - t->lo, n = s->hi - s->lo;
    double* N = (double*)malloc((size_t)(7 * m * n) * sizeof(double));
    double e[7];
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) {
            kernel_entry(h, t->lo + i, s->lo + j, e);
            for (int v = 0; v < 7; ++v) N[(v * m + i) * n + j] = e[v];
        }
    h->Nf[b] = N;
    h->near_done[b] = 1;
}

/* Assemble the listed blocks; a negative count means all blocks of that kind. */
void or_hmat_assemble(void* hp, const int64_t* adm_ids, int64_t nadm_ids, const int64_t* near_ids,
                      int64_t nnear_ids)
{
    or_hmat* h = (or_hmat*)hp;
    int64_t na = nadm_ids < 0 ? h->bl.nadm : nadm_ids;
    int64_t nn = nnear_ids < 0 ? h->bl.nnear : nnear_ids;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < na; ++q) {
        int64_t b = nadm_ids < 0 ? q : adm_ids[q];
        if (!h->adm_done[b]) assemble_adm(h, b);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nn; ++q) {
        int64_t b = nnear_ids < 0 ? q : near_ids[q];
        if (!h->near_done[b]) assemble_near(h, b);
    }
}

int32_t or_hmat_rank(const void* hp, int64_t b, int kern)
{
    const or_hmat* h = (const or_hmat*)hp;
    return h->rank[b * 7 + kern];
}

int32_t or_hmat_aca_flags(const void* hp, int64_t b, int kern)
{
    const or_hmat* h = (const or_hmat*)hp;
    return h->aca_flags[b * 7 + kern];
}

void or_hmat_factors(const void* hp, int64_t b, int kern, double* U, double* Vv)
{
    const or_hmat* h = (const or_hmat*)hp;
    const or_node* t = &h->rnodes[h->bl.adm[b].t];
    const or_node* s = &h->nodes[h->bl.adm[b].s];
    int64_t m = t->hi - t->lo, n = s->hi - s->lo;
    int32_t k = h->rank[b * 7 + kern];
    memcpy(U, h->Uf[b * 7 + kern], (size_t)(m * k) * sizeof(double));
    memcpy(Vv, h->Vf[b * 7 + kern], (size_t)(n * k) * sizeof(double));
}

void or_hmat_near_block(const void* hp, int64_t b, double* out)
{
    const or_hmat* h = (const or_hmat*)hp;
    const or_node* t = &h->rnodes[h->bl.near[b].t];
    const or_node* s = &h->nodes[h->bl.near[b].s];
    int64_t m = t->hi - t->lo, n = s->hi - s->lo;
    memcpy(out, h->Nf[b], (size_t)(7 * m * n) * sizeof(double));
}

/* y = V_h x over the assembled blocks (only the listed ones if lists are
 * given), Eq. (Vh): y_a(i) += c1 sum_j V_Delta[i,j] x_a(j) + c2 sum_{j,b} V_ab[i,j] x_b(j),
 * with c1 = (1+nu)(3-4nu)/(2E(1-nu)) and c2 = (1+nu)/(2E(1-nu)).  Low-rank
 * blocks apply U (V^T x).  x is (nrhs, 3M), y (nrhs, 3 Mr) in original order,
 * dof 3 i + a (Mr = M unless rows are the points of ~V_h).
 * Per block row, blocks are summed in list order.  A negative count means all
 * blocks of that kind; blocks that were not assembled must not be listed. */
static const int kab[3][3] = {{1, 2, 3}, {2, 4, 5}, {3, 5, 6}};

/* The same product with the coefficients of Eq. (Vh) given directly:
 * y_a += c1 V_Delta x_a + c2 sum_b V_ab x_b.  Section 4.2's double layer
 * applies the single layer's blocks with c1 = (1-2nu)/(2(1-nu)) and
 * c2 = 1/(2(1-nu)) (Eq. (Kh), -V_Delta T_h + E/(1+nu) V_h T_h). */
void or_hmat_matvec_c(const void* hp, double c1, double c2, const double* x, double* y,
                      int64_t nrhs, const int64_t* adm_ids, int64_t nadm_ids,
                      const int64_t* near_ids, int64_t nnear_ids);

void or_hmat_matvec(const void* hp, double E, double nu, const double* x, double* y,
                    int64_t nrhs, const int64_t* adm_ids, int64_t nadm_ids,
                    const int64_t* near_ids, int64_t nnear_ids)
{
    double c1 = (1.0 + nu) * (3.0 - 4.0 * nu) / (2.0 * E * (1.0 - nu));
    double c2 = (1.0 + nu) / (2.0 * E * (1.0 - nu));
    or_hmat_matvec_c(hp, c1, c2, x, y, nrhs, adm_ids, nadm_ids, near_ids, nnear_ids);
}

void or_hmat_matvec_c(const void* hp, double c1, double c2, const double* x, double* y,
                      int64_t nrhs, const int64_t* adm_ids, int64_t nadm_ids,
                      const int64_t* near_ids, int64_t nnear_ids)
{
    const or_hmat* h = (const or_hmat*)hp;
    int64_t M = h->M, Mr = h->Mr;
    int64_t na = nadm_ids < 0 ? h->bl.nadm : nadm_ids;
    int64_t nn = nnear_ids < 0 ? h->bl.nnear : nnear_ids;
    if (nadm_ids < 0) adm_ids = NULL;
    if (nnear_ids < 0) near_ids = NULL;
    for (int64_t q = 0; q < nrhs * 3 * Mr; ++q) y[q] = 0.0;
    /* process blocks grouped by row-cluster node id so that threads own rows */
    int64_t nnod = h->nrnodes;
    int64_t* cnt = (int64_t*)calloc((size_t)(nnod + 1), sizeof(int64_t));
    for (int64_t q = 0; q < na; ++q) cnt[h->bl.adm[adm_ids ? adm_ids[q] : q].t + 1]++;
    int64_t* ncnt = (int64_t*)calloc((size_t)(nnod + 1), sizeof(int64_t));
    for (int64_t q = 0; q < nn; ++q) ncnt[h->bl.near[near_ids ? near_ids[q] : q].t + 1]++;
    for (int64_t n = 0; n < nnod; ++n) {
        cnt[n + 1] += cnt[n];
        ncnt[n + 1] += ncnt[n];
    }
    int64_t* ord = (int64_t*)malloc((size_t)(na + 1) * sizeof(int64_t));
    int64_t* nord = (int64_t*)malloc((size_t)(nn + 1) * sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)(nnod + 1), sizeof(int64_t));
    for (int64_t q = 0; q < na; ++q) {
        int64_t b = adm_ids ? adm_ids[q] : q;
        int64_t t = h->bl.adm[b].t;
        ord[cnt[t] + fill[t]++] = b;
    }
    memset(fill, 0, (size_t)(nnod + 1) * sizeof(int64_t));
    for (int64_t q = 0; q < nn; ++q) {
        int64_t b = near_ids ? near_ids[q] : q;
        int64_t t = h->bl.near[b].t;
        nord[ncnt[t] + fill[t]++] = b;
    }
    /* Each level's row clusters are disjoint, so levels run one after the
     * other and the clusters of one level in parallel. */
    int32_t maxlev = 0;
    for (int64_t n = 0; n < nnod; ++n)
        if (h->rnodes[n].level > maxlev) maxlev = h->rnodes[n].level;
    for (int32_t lev = 0; lev <= maxlev; ++lev) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t tn = 0; tn < nnod; ++tn) {
            const or_node* t = &h->rnodes[tn];
            if (t->level != lev) continue;
            int64_t m = t->hi - t->lo;
            double* z = (double*)malloc((size_t)(3 * (h->kmax + 1)) * sizeof(double));
            for (int64_t r = 0; r < nrhs; ++r) {
                const double* xr = x + r * 3 * M;
                double* yr = y + r * 3 * Mr;
                for (int64_t q = cnt[tn]; q < cnt[tn + 1]; ++q) {
                    int64_t b = ord[q];
                    const or_node* s = &h->nodes[h->bl.adm[b].s];
                    int64_t n = s->hi - s->lo;
                    for (int kern = 0; kern < 7; ++kern) {
                        int32_t k = h->rank[b * 7 + kern];
                        const double* U = h->Uf[b * 7 + kern];
                        const double* Vv = h->Vf[b * 7 + kern];
                        /* z_c = V^T x_c(s) for the three components */
                        for (int32_t l = 0; l < k; ++l)
                            for (int c = 0; c < 3; ++c) {
                                double sacc = 0.0;
                                for (int64_t j = 0; j < n; ++j)
                                    sacc += Vv[l * n + j] * xr[3 * h->perm[s->lo + j] + c];
                                z[3 * l + c] = sacc;
                            }
                        for (int64_t i = 0; i < m; ++i) {
                            double* yi = yr + 3 * h->rperm[t->lo + i];
                            for (int a = 0; a < 3; ++a) {
                                double sacc = 0.0;
                                if (kern == 0) {
                                    for (int32_t l = 0; l < k; ++l) sacc += U[l * m + i] * z[3 * l + a];
                                    yi[a] += c1 * sacc;
                                } else {
                                    /* kernel (p,q) contributes to y_p with x_q and to y_q with x_p */
                                    for (int b2 = 0; b2 < 3; ++b2) {
                                        if (kab[a][b2] != kern) continue;
                                        for (int32_t l = 0; l < k; ++l)
                                            sacc += U[l * m + i] * z[3 * l + b2];
                                    }
                                    yi[a] += c2 * sacc;
                                }
                            }
                        }
                    }
                }
                for (int64_t q = ncnt[tn]; q < ncnt[tn + 1]; ++q) {
                    int64_t b = nord[q];
                    const or_node* s = &h->nodes[h->bl.near[b].s];
                    int64_t n = s->hi - s->lo;
                    const double* N = h->Nf[b];
                    for (int64_t i = 0; i < m; ++i) {
                        double* yi = yr + 3 * h->rperm[t->lo + i];
                        for (int64_t j = 0; j < n; ++j) {
                            const double* xj = xr + 3 * h->perm[s->lo + j];
                            double vd = N[(0 * m + i) * n + j];
                            for (int a = 0; a < 3; ++a) {
                                double sacc = c1 * vd * xj[a];
                                for (int b2 = 0; b2 < 3; ++b2)
                                    sacc += c2 * N[(kab[a][b2] * m + i) * n + j] * xj[b2];
                                yi[a] += sacc;
                            }
                        }
                    }
                }
            }
            free(z);
        }
    }
    free(cnt);
    free(ncnt);
    free(ord);
    free(nord);
    free(fill);
}

int32_t or_num_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the later parallel regions started from the calling thread
 * (OpenMP); the arithmetic and its order do not depend on it.  n < 1 is
 * ignored. */
void or_set_num_threads(int32_t n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads((int)n);
#else
    (void)n;
#endif
}
