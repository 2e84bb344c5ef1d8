/*
 * FP64 CPU oracle for differentiable voxelization by the generalized winding number.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * statement of what the CUDA path computes. Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the product never does.
 * It shares no code, header, table or constant with the CUDA sources.
 *
 * Every function follows one passage of the paper:
 *   atan2_table          Eq. (8), the ATAN2 case table
 *   half_solid_angle     Algorithm 1 loop body with Eq. (7): normalize e_j,
 *                        alpha = det(e0,e1,e2), beta = 1 + sum of <e_i,e_j>
 *   orc_solid_angle      Eq. (7) read as Omega = 2 * ATAN2(alpha, beta)
 *   orc_winding          Eq. (5) / Algorithm 1: W(q) = (1/4pi) sum_f Omega_f(q)
 *   orc_grid_queries     §3: cell-centred voxel grid over a box
 *   orc_grid_points      the same centres for selected cells only
 *   orc_winding_grad     derivative of Eq. (5)+(7) by the chain rule through
 *                        the normalized vectors e_j (the paper claims
 *                        differentiability, §1 and §2.4, but prints no formula)
 *   orc_vertex_grad_subset   the same derivative for selected vertices only
 *   orc_winding_grad_scale   per vertex, sum over incident faces of |face contribution|
 *   orc_point_mesh_distance   exact point-to-triangle Euclidean distance
 *   orc_fd_vertex_grad   central finite differences of Eq. (5) in FP64
 *   orc_dipole_winding   Eq. (4), the naive dipole discretization (§2.4)
 *   orc_ray_winding_grid the winding number of a CLOSED mesh on a grid by signed ray
 *                        crossings (Eq. (3)): a check of Eq. (5) that evaluates no solid angle
 *
 * Readings of the paper used here (each is pinned by a test):
 *   - Eq. (7) prints arctan and no factor 2; Algorithm 1 adds ATAN2(alpha, beta).
 *     The half-angle identity tan(Omega/2) = alpha/beta gives Omega = 2 ATAN2,
 *     hence W = (1/2pi) sum ATAN2(alpha, beta).
 *   - A vertex that coincides with q leaves e_j undefined; the face then
 *     contributes ATAN2(0, 0) = 0 (the last case of Eq. (8)).
 *   - Faces counter-clockwise seen from outside give W = +1 inside.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Eq. (8): ATAN2 exactly as the table states it, case by case. */
double atan2_table(double y, double x) {
    if (x > 0) return atan(y / x);
    if (x < 0 && y >= 0) return atan(y / x) + ORC_PI;
    if (x < 0 && y < 0) return atan(y / x) - ORC_PI;
    if (x == 0 && y > 0) return ORC_PI / 2;
    if (x == 0 && y < 0) return -ORC_PI / 2;
    return 0.0;
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double *a, const double *b, double *out) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Algorithm 1, loop body, with Eq. (7): returns ATAN2(alpha, beta) = Omega / 2. */
static double half_solid_angle(const double *v0, const double *v1, const double *v2, const double *q) {
    const double *v[3] = {v0, v1, v2};
    double e[3][3];
    for (int j = 0; j < 3; ++j) {
        double r[3] = {v[j][0] - q[0], v[j][1] - q[1], v[j][2] - q[2]};
        double len = sqrt(dot3(r, r));
        if (len == 0.0) return 0.0; /* ATAN2(0,0) reading for a coincident vertex */
        for (int k = 0; k < 3; ++k) e[j][k] = r[k] / len;
    }
    double c12[3];
    cross3(e[1], e[2], c12);
    double alpha = dot3(e[0], c12);                                   /* det(e0, e1, e2) */
    double beta = 1.0 + dot3(e[0], e[1]) + dot3(e[1], e[2]) + dot3(e[2], e[0]);
    return atan2_table(alpha, beta);
}

/* Eq. (7): solid angle of one triangle seen from q. */
double orc_solid_angle(const double *v0, const double *v1, const double *v2, const double *q) {
    return 2.0 * half_solid_angle(v0, v1, v2, q);
}

static const double *vtx(const double *V, const int32_t *F, int64_t f, int k) { return V + 3 * (int64_t)F[3 * f + k]; }

/* Eq. (5) / Algorithm 1: for every query, sum over every face in input order. */
void orc_winding(const double *V, int64_t nv, const int32_t *F, int64_t nf, const double *Q, int64_t nq,
                 double *w_out, int nthreads) {
    (void)nv;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nq; ++i) {
        double s = 0.0;
        for (int64_t f = 0; f < nf; ++f) s += half_solid_angle(vtx(V, F, f, 0), vtx(V, F, f, 1), vtx(V, F, f, 2), Q + 3 * i);
        w_out[i] = s / (2.0 * ORC_PI); /* (1/4pi) * sum of 2*ATAN2 */
    }
}

/* §3: voxel centres of an n[0] x n[1] x n[2] grid over [lo, hi], x fastest.
 * The box corners arrive as float (the library's grid record) and are widened to double. */
/* Centre of cell (ix, iy, iz): lo + (i + 1/2) h per axis. */
static void cell_centre(const float *lo, const double *h, int64_t ix, int64_t iy, int64_t iz, double *out) {
    out[0] = (double)lo[0] + ((double)ix + 0.5) * h[0];
    out[1] = (double)lo[1] + ((double)iy + 0.5) * h[1];
    out[2] = (double)lo[2] + ((double)iz + 0.5) * h[2];
}

void orc_grid_queries(const float *lo, const float *hi, const int32_t *n, double *out) {
    double h[3];
    for (int k = 0; k < 3; ++k) h[k] = ((double)hi[k] - (double)lo[k]) / (double)n[k];
    int64_t idx = 0;
    for (int32_t iz = 0; iz < n[2]; ++iz)
        for (int32_t iy = 0; iy < n[1]; ++iy)
            for (int32_t ix = 0; ix < n[0]; ++ix) {
                cell_centre(lo, h, ix, iy, iz, out + 3 * idx);
                ++idx;
            }
}

/* The same cell centres for m selected cells, given by their linear index
 * (iz * n[1] + iy) * n[0] + ix (x fastest), so that a sample of a grid too large
 * to list can be evaluated. */
void orc_grid_points(const float *lo, const float *hi, const int32_t *n, const int64_t *cells, int64_t m,
                     double *out) {
    double h[3];
    for (int k = 0; k < 3; ++k) h[k] = ((double)hi[k] - (double)lo[k]) / (double)n[k];
    for (int64_t j = 0; j < m; ++j) {
        const int64_t c = cells[j];
        cell_centre(lo, h, c % n[0], (c / n[0]) % n[1], c / ((int64_t)n[0] * n[1]), out + 3 * j);
    }
}

/* Gradient of W(q) with respect to the three vertices of one face, chain rule
 * through the normalized vectors of Eq. (7):
 *   Omega = 2 ATAN2(alpha, beta)
 *   dOmega/dalpha = 2 beta / (alpha^2 + beta^2),  dOmega/dbeta = -2 alpha / (alpha^2 + beta^2)
 *   dalpha/de0 = e1 x e2, dalpha/de1 = e2 x e0, dalpha/de2 = e0 x e1
 *   dbeta/de_j = sum of the other two e's
 *   de_j/dv_j  = (I - e_j e_j^T) / ||v_j - q||
 * Adds scale * dOmega/dv_j to g[3j..3j+2]. Faces touching q contribute nothing. */
static void face_grad_add(const double *v0, const double *v1, const double *v2, const double *q, double scale,
                          double *g) {
    const double *v[3] = {v0, v1, v2};
    double e[3][3], len[3];
    for (int j = 0; j < 3; ++j) {
        double r[3] = {v[j][0] - q[0], v[j][1] - q[1], v[j][2] - q[2]};
        len[j] = sqrt(dot3(r, r));
        if (len[j] == 0.0) return;
        for (int k = 0; k < 3; ++k) e[j][k] = r[k] / len[j];
    }
    double c12[3], c20[3], c01[3];
    cross3(e[1], e[2], c12);
    cross3(e[2], e[0], c20);
    cross3(e[0], e[1], c01);
    double alpha = dot3(e[0], c12);
    double beta = 1.0 + dot3(e[0], e[1]) + dot3(e[1], e[2]) + dot3(e[2], e[0]);
    double den = alpha * alpha + beta * beta;
    if (den == 0.0) return;
    double da = 2.0 * beta / den, db = -2.0 * alpha / den;
    const double *ga[3] = {c12, c20, c01};
    for (int j = 0; j < 3; ++j) {
        const double *o1 = e[(j + 1) % 3], *o2 = e[(j + 2) % 3];
        double t[3];
        for (int k = 0; k < 3; ++k) t[k] = da * ga[j][k] + db * (o1[k] + o2[k]);
        double et = dot3(e[j], t);
        for (int k = 0; k < 3; ++k) g[3 * j + k] += scale * (t[k] - e[j][k] * et) / len[j];
    }
}

/* dL/dV = sum_q upstream[q] * dW(q)/dV, W from Eq. (5). Parallel over faces,
 * FP64 sums over queries in order, then a serial scatter to the vertices. */
void orc_winding_grad(const double *V, int64_t nv, const int32_t *F, int64_t nf, const double *Q, int64_t nq,
                      const double *upstream, double *dV_out, int nthreads) {
    set_threads(nthreads);
    double *fg = (double *)calloc((size_t)nf * 9, sizeof(double));
    if (!fg) return;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t f = 0; f < nf; ++f) {
        double g[9] = {0};
        for (int64_t i = 0; i < nq; ++i)
            face_grad_add(vtx(V, F, f, 0), vtx(V, F, f, 1), vtx(V, F, f, 2), Q + 3 * i, upstream[i] / (4.0 * ORC_PI), g);
        memcpy(fg + 9 * f, g, sizeof(g));
    }
    memset(dV_out, 0, sizeof(double) * 3 * (size_t)nv);
    for (int64_t f = 0; f < nf; ++f)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) dV_out[3 * (int64_t)F[3 * f + j] + k] += fg[9 * f + 3 * j + k];
    free(fg);
}

/* Magnitude scale of the per-vertex gradient sums: for every vertex, the sum over its
 * incident faces of the Euclidean norm of that face's contribution (same per-face sums as
 * orc_winding_grad). A vertex whose faces' contributions cancel (on a closed part of a mesh
 * the exact result is 0) can only be compared to a tolerance relative to this scale. */
void orc_winding_grad_scale(const double *V, int64_t nv, const int32_t *F, int64_t nf, const double *Q, int64_t nq,
                            const double *upstream, double *scale_out, int nthreads) {
    set_threads(nthreads);
    double *fg = (double *)calloc((size_t)nf * 9, sizeof(double));
    if (!fg) return;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t f = 0; f < nf; ++f) {
        double g[9] = {0};
        for (int64_t i = 0; i < nq; ++i)
            face_grad_add(vtx(V, F, f, 0), vtx(V, F, f, 1), vtx(V, F, f, 2), Q + 3 * i, upstream[i] / (4.0 * ORC_PI), g);
        memcpy(fg + 9 * f, g, sizeof(g));
    }
    memset(scale_out, 0, sizeof(double) * (size_t)nv);
    for (int64_t f = 0; f < nf; ++f)
        for (int j = 0; j < 3; ++j) {
            const double *c = fg + 9 * f + 3 * j;
            scale_out[F[3 * f + j]] += sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        }
    free(fg);
}

/* The same derivative as orc_winding_grad, for selected vertices only: sums over
 * every query and over the faces incident to each selected vertex. out is [nvid, 3]. */
void orc_vertex_grad_subset(const double *V, int64_t nv, const int32_t *F, int64_t nf, const double *Q, int64_t nq,
                            const double *upstream, const int64_t *vids, int64_t nvid, double *out, int nthreads) {
    (void)nv;
    set_threads(nthreads);
    int64_t *inc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nf > 0 ? nf : 1));
    int *corner = (int *)malloc(sizeof(int) * (size_t)(nf > 0 ? nf : 1));
    if (!inc || !corner) {
        free(inc);
        free(corner);
        return;
    }
    for (int64_t t = 0; t < nvid; ++t) {
        int64_t vid = vids[t], ninc = 0;
        for (int64_t f = 0; f < nf; ++f)
            for (int j = 0; j < 3; ++j)
                if (F[3 * f + j] == vid) {
                    inc[ninc] = f;
                    corner[ninc++] = j;
                }
        double s0 = 0, s1 = 0, s2 = 0;
#pragma omp parallel for reduction(+ : s0, s1, s2) schedule(dynamic, 256)
        for (int64_t i = 0; i < nq; ++i) {
            for (int64_t m = 0; m < ninc; ++m) {
                int64_t f = inc[m];
                double g[9] = {0};
                face_grad_add(vtx(V, F, f, 0), vtx(V, F, f, 1), vtx(V, F, f, 2), Q + 3 * i, upstream[i] / (4.0 * ORC_PI),
                              g);
                s0 += g[3 * corner[m]];
                s1 += g[3 * corner[m] + 1];
                s2 += g[3 * corner[m] + 2];
            }
        }
        out[3 * t] = s0;
        out[3 * t + 1] = s1;
        out[3 * t + 2] = s2;
    }
    free(inc);
    free(corner);
}

/* Distance from p to the segment [a, b]. */
static double seg_dist(const double *p, const double *a, const double *b) {
    double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    double L = dot3(ab, ab);
    double t = L > 0 ? dot3(ap, ab) / L : 0.0;
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    double d[3] = {ap[0] - t * ab[0], ap[1] - t * ab[1], ap[2] - t * ab[2]};
    return sqrt(dot3(d, d));
}

/* Exact Euclidean distance from p to triangle (a, b, c): if the orthogonal
 * projection of p onto the plane lies inside the triangle, the distance is
 * the plane distance; otherwise the nearest point is on one of the edges. */
static double tri_dist(const double *p, const double *a, const double *b, const double *c) {
    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double n[3];
    cross3(e1, e2, n);
    double nn = dot3(n, n);
    if (nn > 0) {
        double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
        double s = dot3(ap, n) / nn;                    /* signed offset along n */
        double x[3] = {ap[0] - s * n[0], ap[1] - s * n[1], ap[2] - s * n[2]}; /* projection - a */
        /* barycentric coordinates of the projection from sub-triangle areas */
        double c1[3], c2[3];
        cross3(x, e2, c1);
        cross3(e1, x, c2);
        double u = dot3(c1, n) / nn, v = dot3(c2, n) / nn;
        if (u >= 0 && v >= 0 && u + v <= 1) return fabs(s) * sqrt(nn);
    }
    double d0 = seg_dist(p, a, b), d1 = seg_dist(p, b, c), d2 = seg_dist(p, c, a);
    double d = d0 < d1 ? d0 : d1;
    return d < d2 ? d : d2;
}

void orc_point_mesh_distance(const double *V, int64_t nv, const int32_t *F, int64_t nf, const double *Q, int64_t nq,
                             double *d_out, int nthreads) {
    (void)nv;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nq; ++i) {
        double best = INFINITY;
        for (int64_t f = 0; f < nf; ++f) {
            double d = tri_dist(Q + 3 * i, vtx(V, F, f, 0), vtx(V, F, f, 1), vtx(V, F, f, 2));
            if (d < best) best = d;
        }
        d_out[i] = best;
    }
}

/* Central differences of L = sum_q upstream[q] W(q) with respect to selected
 * vertex coordinates, step h, in FP64. Only faces incident to the perturbed
 * vertex change W, so only those are re-evaluated. out is [nvid, 3]. */
void orc_fd_vertex_grad(const double *V, int64_t nv, const int32_t *F, int64_t nf, const double *Q, int64_t nq,
                        const double *upstream, const int64_t *vids, int64_t nvid, double h, double *out,
                        int nthreads) {
    (void)nv;
    set_threads(nthreads);
    int64_t *inc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nf > 0 ? nf : 1));
    if (!inc) return;
    for (int64_t t = 0; t < nvid; ++t) {
        int64_t vid = vids[t], ninc = 0;
        for (int64_t f = 0; f < nf; ++f)
            if (F[3 * f] == vid || F[3 * f + 1] == vid || F[3 * f + 2] == vid) inc[ninc++] = f;
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(dynamic, 64)
            for (int64_t i = 0; i < nq; ++i) {
                double acc = 0.0;
                for (int64_t m = 0; m < ninc; ++m) {
                    int64_t f = inc[m];
                    double p[3][3];
                    for (int j = 0; j < 3; ++j)
                        for (int c = 0; c < 3; ++c) p[j][c] = V[3 * (int64_t)F[3 * f + j] + c];
                    double plus = 0, minus = 0;
                    for (int sgn = 0; sgn < 2; ++sgn) {
                        double pp[3][3];
                        memcpy(pp, p, sizeof(p));
                        for (int j = 0; j < 3; ++j)
                            if (F[3 * f + j] == vid) pp[j][k] += sgn ? -h : h;
                        double a = half_solid_angle(pp[0], pp[1], pp[2], Q + 3 * i);
                        if (sgn) minus = a; else plus = a;
                    }
                    acc += plus - minus;
                }
                s += upstream[i] * acc;
            }
            out[3 * t + k] = s / (2.0 * ORC_PI) / (2.0 * h);
        }
    }
    free(inc);
}

/* Eq. (4): W(q) ~ (1/4pi) sum_i <n_i, E_q(c_i)> Delta_i with E_q(x) = (x - q)/||x - q||^3,
 * c_i the face centroid, n_i the unit outward normal, Delta_i the face area. */
void orc_dipole_winding(const double *V, int64_t nv, const int32_t *F, int64_t nf, const double *Q, int64_t nq,
                        double *w_out, int nthreads) {
    (void)nv;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nq; ++i) {
        double s = 0.0;
        for (int64_t f = 0; f < nf; ++f) {
            const double *a = vtx(V, F, f, 0), *b = vtx(V, F, f, 1), *c = vtx(V, F, f, 2);
            double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
            double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
            double m[3];
            cross3(e1, e2, m);                 /* m = 2 * area * unit normal */
            double area = 0.5 * sqrt(dot3(m, m));
            if (area == 0.0) continue;
            double nrm[3] = {m[0] / (2 * area), m[1] / (2 * area), m[2] / (2 * area)};
            double x[3];
            for (int k = 0; k < 3; ++k) x[k] = (a[k] + b[k] + c[k]) / 3.0 - Q[3 * i + k];
            double r = sqrt(dot3(x, x));
            if (r == 0.0) continue;
            s += dot3(nrm, x) / (r * r * r) * area;
        }
        w_out[i] = s / (4.0 * ORC_PI);
    }
}

/* ---------------------------------------------------------------------------------------------
 * Winding number of a CLOSED, consistently oriented mesh at every cell centre of a grid, by
 * counting signed crossings of rays (an independent check of Eq. (5) / Algorithm 1 that never
 * evaluates a solid angle). For a closed surface and q off it, the winding number equals the
 * signed number of times a ray from q crosses the surface (Eq. (3): the flux of E_q through the
 * closed surface is 1 inside and 0 outside; a ray leaving the enclosed volume crosses a face
 * whose outward normal points along the ray). Each row of cells (fixed y, z) gets one ray along
 * +x: for every face whose projection onto the yz plane contains (y, z), the crossing abscissa
 * x_c (barycentric interpolation) counts +1 if the face normal n = (v1 - v0) x (v2 - v0) has
 * n_x > 0 and -1 if n_x < 0, and a cell with centre x gets the sum over crossings with x_c > x.
 * A count is marked undecided (amb_out = 1) when its row passes within a relative barycentric
 * distance eps_bary of an edge or vertex of a face in the projection, or when the centre lies
 * within eps_x of a crossing (q on or next to the surface). Grid layout as orc_grid_queries.
 */
typedef struct {
    double x;
    int sign;
} orc_crossing;

static int orc_crossing_cmp(const void *a, const void *b) {
    const double xa = ((const orc_crossing *)a)->x, xb = ((const orc_crossing *)b)->x;
    return (xa > xb) - (xa < xb);
}

/* Rows j with centre lo + (j + 0.5) h inside [a, b], clamped to [0, n - 1]. */
static void orc_row_range(double a, double b, double lo, double h, int32_t n, int64_t *j0, int64_t *j1) {
    double s = ceil((a - lo) / h - 0.5), e = floor((b - lo) / h - 0.5);
    if (s < 0) s = 0;
    if (e > n - 1) e = n - 1;
    *j0 = (int64_t)s;
    *j1 = (int64_t)e;
}

int orc_ray_winding_grid(const double *V, int64_t nv, const int32_t *F, int64_t nf, const float *lo, const float *hi,
                         const int32_t *n, double eps_bary, double eps_x, int32_t *w_out, uint8_t *amb_out,
                         int nthreads) {
    (void)nv;
    set_threads(nthreads);
    double h[3];
    for (int k = 0; k < 3; ++k) h[k] = ((double)hi[k] - (double)lo[k]) / (double)n[k];
    const int64_t nrows = (int64_t)n[1] * n[2];
    int64_t *count = (int64_t *)calloc((size_t)nrows + 1, sizeof(int64_t));
    uint8_t *row_amb = (uint8_t *)calloc((size_t)nrows, 1);
    if (!count || !row_amb) {
        free(count);
        free(row_amb);
        return 1;
    }
    /* two passes over the faces: count the crossings of each row, then store them */
    orc_crossing *cr = NULL;
    int64_t *fill = NULL;
    for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t f = 0; f < nf; ++f) {
            const double *a = vtx(V, F, f, 0), *b = vtx(V, F, f, 1), *c = vtx(V, F, f, 2);
            const double d = (b[1] - a[1]) * (c[2] - a[2]) - (c[1] - a[1]) * (b[2] - a[2]); /* n_x */
            if (d == 0.0) continue; /* seen edge-on from the rays: its edges decide */
            const double ymin = fmin(a[1], fmin(b[1], c[1])), ymax = fmax(a[1], fmax(b[1], c[1]));
            const double zmin = fmin(a[2], fmin(b[2], c[2])), zmax = fmax(a[2], fmax(b[2], c[2]));
            const double gy = 1e-9 * (1.0 + ymax - ymin), gz = 1e-9 * (1.0 + zmax - zmin);
            int64_t y0, y1, z0, z1;
            orc_row_range(ymin - gy, ymax + gy, lo[1], h[1], n[1], &y0, &y1);
            orc_row_range(zmin - gz, zmax + gz, lo[2], h[2], n[2], &z0, &z1);
            for (int64_t iz = z0; iz <= z1; ++iz)
                for (int64_t iy = y0; iy <= y1; ++iy) {
                    const double y = (double)lo[1] + ((double)iy + 0.5) * h[1];
                    const double z = (double)lo[2] + ((double)iz + 0.5) * h[2];
                    const double l1 = ((y - a[1]) * (c[2] - a[2]) - (c[1] - a[1]) * (z - a[2])) / d;
                    const double l2 = ((b[1] - a[1]) * (z - a[2]) - (y - a[1]) * (b[2] - a[2])) / d;
                    const double l0 = 1.0 - l1 - l2;
                    const double m = fmin(l0, fmin(l1, l2));
                    const int64_t row = iz * n[1] + iy;
                    if (m > eps_bary) {
                        if (pass == 0) {
#pragma omp atomic
                            count[row + 1] += 1;
                        } else {
                            int64_t slot;
#pragma omp atomic capture
                            slot = fill[row]++;
                            cr[slot].x = l0 * a[0] + l1 * b[0] + l2 * c[0];
                            cr[slot].sign = d > 0 ? 1 : -1;
                        }
                    } else if (pass == 0 && m > -eps_bary) {
                        row_amb[row] = 1; /* the ray grazes an edge or a vertex */
                    }
                }
        }
        if (pass == 0) {
            for (int64_t r = 0; r < nrows; ++r) count[r + 1] += count[r];
            cr = (orc_crossing *)malloc(sizeof(orc_crossing) * (size_t)(count[nrows] > 0 ? count[nrows] : 1));
            fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nrows);
            if (!cr || !fill) {
                free(cr);
                free(fill);
                free(count);
                free(row_amb);
                return 1;
            }
            for (int64_t r = 0; r < nrows; ++r) fill[r] = count[r];
        }
    }
    /* per row: crossings in x order, then each centre counts those beyond it */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nrows; ++r) {
        orc_crossing *c = cr + count[r];
        const int64_t m = count[r + 1] - count[r];
        qsort(c, (size_t)m, sizeof(orc_crossing), orc_crossing_cmp);
        int64_t k = m; /* crossings c[k..m) lie beyond the current centre */
        int32_t beyond = 0;
        for (int64_t ix = n[0] - 1; ix >= 0; --ix) {
            const double x = (double)lo[0] + (0.5 + (double)ix) * h[0];
            while (k > 0 && c[k - 1].x > x) beyond += c[--k].sign;
            int near = 0;
            if (k > 0 && x - c[k - 1].x <= eps_x) near = 1;
            if (k < m && c[k].x - x <= eps_x) near = 1;
            const int64_t idx = r * n[0] + ix;
            w_out[idx] = beyond;
            amb_out[idx] = (uint8_t)(row_amb[r] || near);
        }
    }
    free(cr);
    free(fill);
    free(count);
    free(row_amb);
    return 0;
}
