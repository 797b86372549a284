/*
 * bem_oracle.c -- plain FP64 reference for the P1 Galerkin boundary operators
 * of the Helmholtz transmission problem (arXiv 1910.01011).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct oracle
 * the CUDA library is checked against.  Only tests/, the smoke check and the
 * CPU-baseline leg of bench.py may load it.  It shares no code with the CUDA
 * path.
 *
 * What it computes (paper App. A, eqs. SLP/DLP/ADJDLP/HYP; Sec. 2.3 eq.
 * Galerkin_disc_lhs): for a test surface X and a trial surface Y, the
 * Galerkin matrices of the four boundary integral operators with continuous
 * piecewise-linear (P1) test and trial functions,
 *
 *   V [r][q]  = int_X int_Y phi_r(x) G(x,y)          phi_q(y)
 *   K [r][q]  = int_X int_Y phi_r(x) dG/dn_y(x,y)    phi_q(y)
 *   K'[r][q]  = int_X int_Y phi_r(x) dG/dn_x(x,y)    phi_q(y)
 *   W [r][q]  = int_X int_Y G(x,y) [curl phi_r(x).curl phi_q(y)
 *                                  - k^2 (n_x.n_y) phi_r(x) phi_q(y)]
 *
 * with G(x,y) = exp(ik|x-y|)/(4 pi |x-y|) (App. A eq. green_func).  The W
 * line is the standard integration-by-parts (Maue) form of
 * W = -d/dn_x int dG/dn_y (App. A eq. HYP); the paper states no weak form.
 *
 * Quadrature (the paper defers to its BEM library; the reading is fixed in
 * the design notes and shared with the CUDA path as a *rule*, not as code):
 *   - pairs of triangles with no common vertex: a symmetric triangle rule
 *     (the 6-point degree-4 rule, passed in) on both triangles;
 *   - of those, the near pairs, whose centroids are closer than twice the
 *     longer of the two triangles' longest edges: a collapsed Gauss-Legendre
 *     rule on each triangle (the n Gauss-Legendre nodes passed in, in both
 *     directions of the unit square, mapped by s1 = u, s2 = u v with
 *     Jacobian u onto the reference triangle below);
 *   - pairs sharing a vertex, an edge, or identical: the Sauter-Schwab
 *     regularising transformations (Sauter & Schwab, Boundary Element
 *     Methods, Sec. 5.2) with an n-point Gauss-Legendre rule in each of the
 *     four reference directions (nodes passed in).
 *
 * Triangle parametrisation used for the singular rules: reference triangle
 * {0 <= s2 <= s1 <= 1}, x(s) = P0 + s1 (P1 - P0) + s2 (P2 - P1), Jacobian
 * 2|T|, barycentric values (1 - s1, s1 - s2, s2) at vertices (P0, P1, P2).
 * Shared vertices are put first in both triangles (common edge P0P1, common
 * vertex P0).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex zc;

#define REL_NONE 0
#define REL_VERTEX 1
#define REL_EDGE 2
#define REL_SAME 3
#define REL_NEAR 4 /* reported by orc_pair only: no common vertex, but near */

typedef struct {
    double P[3][3];    /* vertex coordinates, local order */
    double n[3];       /* unit outward normal (from the original orientation) */
    double area;
    double curl[3][3]; /* surface curl of the three local P1 functions */
} tri_t;

typedef struct {
    zc V[3][3], K[3][3], Kp[3][3], W[3][3];
} pairmat;

static void sub3(const double *a, const double *b, double *o) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Normal and area from the outward (counter-clockwise) vertex order a,b,c;
 * the vertices are then stored in the local order given by perm. */
static void tri_setup(tri_t *T, const double *V3[3], const int perm[3]) {
    double e1[3], e2[3], c[3];
    sub3(V3[1], V3[0], e1);
    sub3(V3[2], V3[0], e2);
    cross3(e1, e2, c);
    double l = sqrt(dot3(c, c));
    T->area = 0.5 * l;
    for (int i = 0; i < 3; i++) T->n[i] = c[i] / l;
    for (int i = 0; i < 3; i++)
        for (int d = 0; d < 3; d++) T->P[i][d] = V3[perm[i]][d];
    /* curl_G lambda_i = n x grad_G lambda_i = -(edge opposite i, taken
     * counter-clockwise about n)/(2|T|).  Written here via the gradient:
     * grad lambda_i = n x (P_{i+2} - P_{i+1}) / (2|T|) for a CCW triple.
     * For a permuted local order the CCW sense may be reversed, so the
     * gradient is computed from the original CCW order and re-indexed. */
    double g[3][3];
    for (int i = 0; i < 3; i++) {
        double e[3];
        sub3(V3[(i + 2) % 3], V3[(i + 1) % 3], e);
        double t[3];
        cross3(T->n, e, t);
        for (int d = 0; d < 3; d++) g[i][d] = t[d] / (2.0 * T->area);
    }
    for (int i = 0; i < 3; i++) {
        double t[3];
        cross3(T->n, g[perm[i]], t);
        for (int d = 0; d < 3; d++) T->curl[i][d] = t[d];
    }
}

/* Add weight * (kernel contributions at x,y) into M. px, py: P1 values of
 * the local test/trial functions at x and y. */
static void accumulate(pairmat *M, const tri_t *X, const tri_t *Y, const double *x, const double *y,
                       const double *px, const double *py, double w, zc k) {
    double d[3];
    sub3(x, y, d);
    double r = sqrt(dot3(d, d));
    zc G = cexp(I * k * r) / (4.0 * M_PI * r);
    zc dGr = G * (I * k - 1.0 / r) / r; /* (dG/dr) / r */
    zc dGny = dGr * (-dot3(d, Y->n));   /* dG/dn_y = dG/dr (y-x).n_y / r */
    zc dGnx = dGr * dot3(d, X->n);      /* dG/dn_x = dG/dr (x-y).n_x / r */
    double nn = dot3(X->n, Y->n);
    zc k2 = k * k;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double pp = px[i] * py[j];
            M->V[i][j] += w * G * pp;
            M->K[i][j] += w * dGny * pp;
            M->Kp[i][j] += w * dGnx * pp;
            M->W[i][j] += w * G * (dot3(X->curl[i], Y->curl[j]) - k2 * nn * pp);
        }
}

/* Regular rule on both triangles: nq points (l1, l2, weight) with
 * x = P0 + l1 (P1-P0) + l2 (P2-P0), barycentric (1-l1-l2, l1, l2), weights
 * summing to 1 (scaled by the area here). */
static void pair_regular(pairmat *M, const tri_t *X, const tri_t *Y, zc k, int nq, const double *qr) {
    for (int a = 0; a < nq; a++) {
        double l1 = qr[3 * a], l2 = qr[3 * a + 1], wa = qr[3 * a + 2] * X->area;
        double px[3] = {1.0 - l1 - l2, l1, l2}, x[3];
        for (int d = 0; d < 3; d++)
            x[d] = X->P[0][d] + l1 * (X->P[1][d] - X->P[0][d]) + l2 * (X->P[2][d] - X->P[0][d]);
        for (int b = 0; b < nq; b++) {
            double m1 = qr[3 * b], m2 = qr[3 * b + 1], wb = qr[3 * b + 2] * Y->area;
            double py[3] = {1.0 - m1 - m2, m1, m2}, y[3];
            for (int d = 0; d < 3; d++)
                y[d] = Y->P[0][d] + m1 * (Y->P[1][d] - Y->P[0][d]) + m2 * (Y->P[2][d] - Y->P[0][d]);
            accumulate(M, X, Y, x, y, px, py, wa * wb, k);
        }
    }
}

/*
 * Sauter-Schwab transformations.  For a point (xi, e1, e2, e3) of [0,1]^4 and
 * a region index, return the reference points s (test) and t (trial) in
 * {0 <= s2 <= s1 <= 1} and the Jacobian of the map.  Integrating
 * f(s,t) over [0,1]^4 with the Jacobian and summing over regions gives the
 * integral of f over the product of two reference triangles.
 *   identical  (6 regions), common edge on s2 = t2 = 0 (5 regions),
 *   common vertex at s = t = 0 (2 regions).
 */
int orc_ss_nregions(int rel) {
    return rel == REL_SAME ? 6 : rel == REL_EDGE ? 5 : rel == REL_VERTEX ? 2 : 0;
}

void orc_ss_map(int rel, int reg, double xi, double e1, double e2, double e3, double *s, double *t,
                double *jac) {
    if (rel == REL_SAME) {
        *jac = xi * xi * xi * e1 * e1 * e2;
        switch (reg) {
        case 0: s[0] = xi; s[1] = xi * (1 - e1 + e1 * e2); t[0] = xi * (1 - e1 * e2 * e3); t[1] = xi * (1 - e1); break;
        case 1: s[0] = xi * (1 - e1 * e2 * e3); s[1] = xi * (1 - e1); t[0] = xi; t[1] = xi * (1 - e1 + e1 * e2); break;
        case 2: s[0] = xi; s[1] = xi * e1 * (1 - e2 + e2 * e3); t[0] = xi * (1 - e1 * e2); t[1] = xi * e1 * (1 - e2); break;
        case 3: s[0] = xi * (1 - e1 * e2); s[1] = xi * e1 * (1 - e2); t[0] = xi; t[1] = xi * e1 * (1 - e2 + e2 * e3); break;
        case 4: s[0] = xi * (1 - e1 * e2 * e3); s[1] = xi * e1 * (1 - e2 * e3); t[0] = xi; t[1] = xi * e1 * (1 - e2); break;
        default: s[0] = xi; s[1] = xi * e1 * (1 - e2); t[0] = xi * (1 - e1 * e2 * e3); t[1] = xi * e1 * (1 - e2 * e3); break;
        }
    } else if (rel == REL_EDGE) {
        *jac = xi * xi * xi * e1 * e1 * (reg == 0 ? 1.0 : e2);
        switch (reg) {
        case 0: s[0] = xi; s[1] = xi * e1 * e3; t[0] = xi * (1 - e1 * e2); t[1] = xi * e1 * (1 - e2); break;
        case 1: s[0] = xi; s[1] = xi * e1; t[0] = xi * (1 - e1 * e2 * e3); t[1] = xi * e1 * e2 * (1 - e3); break;
        case 2: s[0] = xi * (1 - e1 * e2); s[1] = xi * e1 * (1 - e2); t[0] = xi; t[1] = xi * e1 * e2 * e3; break;
        case 3: s[0] = xi * (1 - e1 * e2 * e3); s[1] = xi * e1 * e2 * (1 - e3); t[0] = xi; t[1] = xi * e1; break;
        default: s[0] = xi * (1 - e1 * e2 * e3); s[1] = xi * e1 * (1 - e2 * e3); t[0] = xi; t[1] = xi * e1 * e2; break;
        }
    } else { /* common vertex */
        *jac = xi * xi * xi * e2;
        if (reg == 0) { s[0] = xi; s[1] = xi * e1; t[0] = xi * e2; t[1] = xi * e2 * e3; }
        else { s[0] = xi * e2; s[1] = xi * e2 * e3; t[0] = xi; t[1] = xi * e1; }
    }
}

static void ref_point(const tri_t *T, const double *s, double *x, double *phi) {
    for (int d = 0; d < 3; d++)
        x[d] = T->P[0][d] + s[0] * (T->P[1][d] - T->P[0][d]) + s[1] * (T->P[2][d] - T->P[1][d]);
    phi[0] = 1.0 - s[0];
    phi[1] = s[0] - s[1];
    phi[2] = s[1];
}

static void pair_singular(pairmat *M, const tri_t *X, const tri_t *Y, int rel, zc k, int ng, const double *gl) {
    int nreg = orc_ss_nregions(rel);
    double scale = (2.0 * X->area) * (2.0 * Y->area);
    for (int a = 0; a < ng; a++)
        for (int b = 0; b < ng; b++)
            for (int c = 0; c < ng; c++)
                for (int e = 0; e < ng; e++) {
                    double w = gl[2 * a + 1] * gl[2 * b + 1] * gl[2 * c + 1] * gl[2 * e + 1];
                    for (int reg = 0; reg < nreg; reg++) {
                        double s[2], t[2], jac, x[3], y[3], px[3], py[3];
                        orc_ss_map(rel, reg, gl[2 * a], gl[2 * b], gl[2 * c], gl[2 * e], s, t, &jac);
                        ref_point(X, s, x, px);
                        ref_point(Y, t, y, py);
                        accumulate(M, X, Y, x, y, px, py, w * jac * scale, k);
                    }
                }
}

/* Near pair: centroids closer than twice the longest edge of either triangle
 * (squared distances, vertex coordinates in their original order). */
static int is_near(const double *VX[3], const double *VY[3]) {
    double cx[3], cy[3], h2 = 0.0;
    for (int d = 0; d < 3; d++) {
        cx[d] = (VX[0][d] + VX[1][d] + VX[2][d]) / 3.0;
        cy[d] = (VY[0][d] + VY[1][d] + VY[2][d]) / 3.0;
    }
    for (int i = 0; i < 3; i++) {
        double e[3];
        sub3(VX[(i + 1) % 3], VX[i], e);
        if (dot3(e, e) > h2) h2 = dot3(e, e);
        sub3(VY[(i + 1) % 3], VY[i], e);
        if (dot3(e, e) > h2) h2 = dot3(e, e);
    }
    double c[3];
    sub3(cx, cy, c);
    return dot3(c, c) < 4.0 * h2;
}

/* Near pair: the collapsed Gauss-Legendre rule on both triangles, in the
 * reference parametrisation of the singular rules (Jacobian 2|T| u each). */
static void pair_near(pairmat *M, const tri_t *X, const tri_t *Y, zc k, int ng, const double *gl) {
    const double scale = (2.0 * X->area) * (2.0 * Y->area);
    for (int a = 0; a < ng; a++)
        for (int b = 0; b < ng; b++) {
            const double u = gl[2 * a], s[2] = {u, u * gl[2 * b]};
            const double wx = gl[2 * a + 1] * gl[2 * b + 1] * u;
            double x[3], px[3];
            ref_point(X, s, x, px);
            for (int c = 0; c < ng; c++)
                for (int e = 0; e < ng; e++) {
                    const double v = gl[2 * c], t[2] = {v, v * gl[2 * e]};
                    const double wy = gl[2 * c + 1] * gl[2 * e + 1] * v;
                    double y[3], py[3];
                    ref_point(Y, t, y, py);
                    accumulate(M, X, Y, x, y, px, py, wx * wy * scale, k);
                }
        }
}

/* Relation of two triangles of the same surface from their vertex ids, and
 * local orders that put the shared vertices first (in matching order). */
static int classify(const int *a, const int *b, int pa[3], int pb[3]) {
    int sa[3], sb[3], ns = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            if (a[i] == b[j]) { sa[ns] = i; sb[ns] = j; ns++; }
    if (ns == 3) {
        for (int i = 0; i < 3; i++) { pa[i] = i; pb[i] = sb[i]; }
        /* identical: same geometric order on both sides */
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                if (b[j] == a[i]) pb[i] = j;
        return REL_SAME;
    }
    if (ns == 0) { for (int i = 0; i < 3; i++) { pa[i] = i; pb[i] = i; } return REL_NONE; }
    int ua[3] = {0, 0, 0}, ub[3] = {0, 0, 0};
    for (int m = 0; m < ns; m++) { pa[m] = sa[m]; pb[m] = sb[m]; ua[sa[m]] = 1; ub[sb[m]] = 1; }
    int ia = ns, ib = ns;
    for (int i = 0; i < 3; i++) { if (!ua[i]) pa[ia++] = i; if (!ub[i]) pb[ib++] = i; }
    return ns == 2 ? REL_EDGE : REL_VERTEX;
}

/* Local 3x3 matrices of one pair in the triangles' ORIGINAL local order. */
static void pair_local(pairmat *out, const double *VX[3], const int *ix, const double *VY[3], const int *iy,
                       int same_surface, zc k, int nq, const double *qr, int ng, const double *gl) {
    int pa[3] = {0, 1, 2}, pb[3] = {0, 1, 2};
    int rel = same_surface ? classify(ix, iy, pa, pb) : REL_NONE;
    tri_t X, Y;
    tri_setup(&X, VX, pa);
    tri_setup(&Y, VY, pb);
    pairmat M;
    memset(&M, 0, sizeof M);
    if (rel == REL_NONE && is_near(VX, VY)) pair_near(&M, &X, &Y, k, ng, gl);
    else if (rel == REL_NONE) pair_regular(&M, &X, &Y, k, nq, qr);
    else pair_singular(&M, &X, &Y, rel, k, ng, gl);
    memset(out, 0, sizeof *out);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            out->V[pa[i]][pb[j]] = M.V[i][j];
            out->K[pa[i]][pb[j]] = M.K[i][j];
            out->Kp[pa[i]][pb[j]] = M.Kp[i][j];
            out->W[pa[i]][pb[j]] = M.W[i][j];
        }
}

/* One pair, exported for tests: out = 4 x 3 x 3 complex (V, K, K', W),
 * interleaved (re, im).  rel_out receives the detected relation. */
int orc_pair(const double *vx, const int *ix, const double *vy, const int *iy, int same_surface, double kre,
             double kim, int nq, const double *qr, int ng, const double *gl, double *out, int *rel_out) {
    const double *VX[3] = {vx, vx + 3, vx + 6}, *VY[3] = {vy, vy + 3, vy + 6};
    int pa[3], pb[3];
    *rel_out = same_surface ? classify(ix, iy, pa, pb) : REL_NONE;
    if (*rel_out == REL_NONE && is_near(VX, VY)) *rel_out = REL_NEAR;
    pairmat M;
    pair_local(&M, VX, ix, VY, iy, same_surface, kre + I * kim, nq, qr, ng, gl);
    zc *o = (zc *)out;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            o[0 * 9 + 3 * i + j] = M.V[i][j];
            o[1 * 9 + 3 * i + j] = M.K[i][j];
            o[2 * 9 + 3 * i + j] = M.Kp[i][j];
            o[3 * 9 + 3 * i + j] = M.W[i][j];
        }
    return 0;
}

/*
 * Galerkin rows of V, K, K', W between a test surface X and a trial surface
 * Y at wavenumber k.  rowmap[v] (v a test vertex) is the output row of v or
 * -1 to skip it.  out: 4 blocks (V, K, K', W), each nrows x nvy complex,
 * interleaved (re, im), accumulated into (caller zeroes it).
 * same_surface != 0 means X and Y are the same mesh (vertex ids shared), in
 * which case touching pairs use the singular rules.
 */
int orc_rows(int nvx, const double *vx, int ntx, const int *tx, int nvy, const double *vy, int nty,
             const int *ty, int same_surface, double kre, double kim, int nq, const double *qr, int ng,
             const double *gl, const int *rowmap, int nrows, double *out) {
    (void)nvx;
    zc k = kre + I * kim;
    zc *o = (zc *)out;
    size_t blk = (size_t)nrows * (size_t)nvy;
#pragma omp parallel
    {
        zc *strip = (zc *)calloc((size_t)12 * nvy, sizeof(zc));
#pragma omp for schedule(dynamic, 4)
        for (int a = 0; a < ntx; a++) {
            const int *ia = tx + 3 * a;
            int need = 0;
            for (int i = 0; i < 3; i++) need |= rowmap[ia[i]] >= 0;
            if (!need) continue;
            memset(strip, 0, (size_t)12 * nvy * sizeof(zc));
            const double *VX[3] = {vx + 3 * ia[0], vx + 3 * ia[1], vx + 3 * ia[2]};
            for (int b = 0; b < nty; b++) {
                const int *ib = ty + 3 * b;
                const double *VY[3] = {vy + 3 * ib[0], vy + 3 * ib[1], vy + 3 * ib[2]};
                pairmat M;
                pair_local(&M, VX, ia, VY, ib, same_surface, k, nq, qr, ng, gl);
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) {
                        size_t c = (size_t)ib[j];
                        strip[(0 * 3 + i) * (size_t)nvy + c] += M.V[i][j];
                        strip[(1 * 3 + i) * (size_t)nvy + c] += M.K[i][j];
                        strip[(2 * 3 + i) * (size_t)nvy + c] += M.Kp[i][j];
                        strip[(3 * 3 + i) * (size_t)nvy + c] += M.W[i][j];
                    }
            }
#pragma omp critical
            for (int i = 0; i < 3; i++) {
                int r = rowmap[ia[i]];
                if (r < 0) continue;
                for (int op = 0; op < 4; op++) {
                    zc *dst = o + op * blk + (size_t)r * nvy;
                    const zc *src = strip + (op * 3 + i) * (size_t)nvy;
                    for (int c = 0; c < nvy; c++) dst[c] += src[c];
                }
            }
        }
        free(strip);
    }
    return 0;
}

/* Number of kernel evaluations orc_rows performs for a given row map
 * (regular pairs only: nq*nq per pair), used to report interactions/s. */
long long orc_rows_regular_evals(int ntx, const int *tx, int nty, const int *rowmap, int nq) {
    long long n = 0;
    for (int a = 0; a < ntx; a++) {
        const int *ia = tx + 3 * a;
        int need = 0;
        for (int i = 0; i < 3; i++) need |= rowmap[ia[i]] >= 0;
        if (need) n += (long long)nty * nq * nq;
    }
    return n;
}
