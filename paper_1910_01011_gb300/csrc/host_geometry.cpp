// host_geometry.cpp -- host-side set-up of the tiled surface data.
//
// * Quadrature (the paper defers quadrature to its BEM library; the reading
//   fixed for this library): the symmetric 6-point degree-4 triangle rule
//   for pairs of triangles without a common vertex, derived below from its
//   moment equations by Newton's method; Sauter-Schwab regularising maps
//   (Sauter & Schwab, Boundary Element Methods, Sec. 5.2) with n-point
//   Gauss-Legendre rules for identical, edge- and vertex-adjacent pairs.
// * P1 Galerkin geometry (paper Sec. 2.3): per triangle the unit normal from
//   the counter-clockwise vertex order, area, the surface curls of the three
//   hat functions (constant on a flat triangle), the rule points and weights.
// * Tiling: per domain, triangles sorted along a Morton curve of their
//   centroids and cut into tiles of TT triangles; points are stored relative
//   to the tile centre.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>

#include "internal.h"

namespace gbem {

// ---------------------------------------------------------------- quadrature

static bool solve4(double A[4][4], double b[4], double x[4]) {
    int piv[4] = {0, 1, 2, 3};
    for (int c = 0; c < 4; c++) {
        int best = c;
        for (int r = c + 1; r < 4; r++)
            if (std::fabs(A[piv[r]][c]) > std::fabs(A[piv[best]][c])) best = r;
        std::swap(piv[c], piv[best]);
        double d = A[piv[c]][c];
        if (d == 0.0) return false;
        for (int r = c + 1; r < 4; r++) {
            double f = A[piv[r]][c] / d;
            for (int k = c; k < 4; k++) A[piv[r]][k] -= f * A[piv[c]][k];
            b[piv[r]] -= f * b[piv[c]];
        }
    }
    for (int c = 3; c >= 0; c--) {
        double s = b[piv[c]];
        for (int k = c + 1; k < 4; k++) s -= A[piv[c]][k] * x[k];
        x[c] = s / A[piv[c]][c];
    }
    return true;
}

// Symmetric rule with orbits (a,a,1-2a), (b,b,1-2b) and weights w1, w2 per
// point.  Exact for degree <= 4 iff exact on the S3-invariant polynomials
// 1, s2, s3, s2^2 of the barycentrics (s2 = sum_{i<j} l_i l_j, s3 = l1 l2 l3),
// whose means over a triangle are 1, 1/4, 1/60, 1/15.
static bool rule6(double out_l1[QP], double out_l2[QP], double out_w[QP]) {
    double a = 0.44, b = 0.09, w1 = 0.22, w2 = 0.11;
    for (int it = 0; it < 100; it++) {
        double s2a = 2 * a - 3 * a * a, s2b = 2 * b - 3 * b * b;
        double s3a = a * a - 2 * a * a * a, s3b = b * b - 2 * b * b * b;
        double ds2a = 2 - 6 * a, ds2b = 2 - 6 * b, ds3a = 2 * a - 6 * a * a, ds3b = 2 * b - 6 * b * b;
        double F[4] = {3 * w1 + 3 * w2 - 1.0, 3 * w1 * s2a + 3 * w2 * s2b - 0.25,
                       3 * w1 * s3a + 3 * w2 * s3b - 1.0 / 60.0,
                       3 * w1 * s2a * s2a + 3 * w2 * s2b * s2b - 1.0 / 15.0};
        double J[4][4] = {{0, 0, 3, 3},
                          {3 * w1 * ds2a, 3 * w2 * ds2b, 3 * s2a, 3 * s2b},
                          {3 * w1 * ds3a, 3 * w2 * ds3b, 3 * s3a, 3 * s3b},
                          {6 * w1 * s2a * ds2a, 6 * w2 * s2b * ds2b, 3 * s2a * s2a, 3 * s2b * s2b}};
        double d[4];
        if (!solve4(J, F, d)) return false;
        a -= d[0]; b -= d[1]; w1 -= d[2]; w2 -= d[3];
        if (std::fabs(d[0]) + std::fabs(d[1]) + std::fabs(d[2]) + std::fabs(d[3]) < 1e-17) break;
    }
    const double orb[2] = {a, b}, wt[2] = {w1, w2};
    int k = 0;
    for (int o = 0; o < 2; o++) {
        double t = orb[o], u = 1 - 2 * t;
        double bary[3][3] = {{t, t, u}, {t, u, t}, {u, t, t}};
        for (int p = 0; p < 3; p++, k++) {
            out_l1[k] = bary[p][1];
            out_l2[k] = bary[p][2];
            out_w[k] = wt[o];
        }
    }
    return std::fabs(a - b) > 0.1;
}

bool gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; i++) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = n == 0 ? 1 : p1, pm = n == 1 ? 1 : p0;
            if (n == 1) { pn = z; pm = 1; }
            dp = n * (z * pn - pm) / (z * z - 1);
            double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[n - 1 - i] = 0.5 * (z + 1);
        w[n - 1 - i] = 1.0 / ((1 - z * z) * dp * dp);  // 2/((1-z^2) P'^2) halved for [0,1]
    }
    return true;
}

// Sauter-Schwab maps: for (xi, e1, e2, e3) in [0,1]^4 and a region, the
// reference points s (test), t (trial) in {0 <= s2 <= s1 <= 1} and the
// Jacobian.  Identical: 6 regions; common edge on s2 = t2 = 0: 5 regions;
// common vertex at the origin: 2 regions.
static void ss_map(int rel, int reg, double xi, double e1, double e2, double e3, double s[2], double t[2]) {
    if (rel == 3) {
        const double a = e1 * e2 * e3, b = e1 * e2;
        switch (reg) {
            case 0: s[0] = xi; s[1] = xi * (1 - e1 + b); t[0] = xi * (1 - a); t[1] = xi * (1 - e1); break;
            case 1: s[0] = xi * (1 - a); s[1] = xi * (1 - e1); t[0] = xi; t[1] = xi * (1 - e1 + b); break;
            case 2: s[0] = xi; s[1] = xi * e1 * (1 - e2 + e2 * e3); t[0] = xi * (1 - b); t[1] = xi * e1 * (1 - e2); break;
            case 3: s[0] = xi * (1 - b); s[1] = xi * e1 * (1 - e2); t[0] = xi; t[1] = xi * e1 * (1 - e2 + e2 * e3); break;
            case 4: s[0] = xi * (1 - a); s[1] = xi * e1 * (1 - e2 * e3); t[0] = xi; t[1] = xi * e1 * (1 - e2); break;
            default: s[0] = xi; s[1] = xi * e1 * (1 - e2); t[0] = xi * (1 - a); t[1] = xi * e1 * (1 - e2 * e3); break;
        }
    } else if (rel == 2) {
        switch (reg) {
            case 0: s[0] = xi; s[1] = xi * e1 * e3; t[0] = xi * (1 - e1 * e2); t[1] = xi * e1 * (1 - e2); break;
            case 1: s[0] = xi; s[1] = xi * e1; t[0] = xi * (1 - e1 * e2 * e3); t[1] = xi * e1 * e2 * (1 - e3); break;
            case 2: s[0] = xi * (1 - e1 * e2); s[1] = xi * e1 * (1 - e2); t[0] = xi; t[1] = xi * e1 * e2 * e3; break;
            case 3: s[0] = xi * (1 - e1 * e2 * e3); s[1] = xi * e1 * e2 * (1 - e3); t[0] = xi; t[1] = xi * e1; break;
            default: s[0] = xi * (1 - e1 * e2 * e3); s[1] = xi * e1 * (1 - e2 * e3); t[0] = xi; t[1] = xi * e1 * e2; break;
        }
    } else {
        if (reg == 0) { s[0] = xi; s[1] = xi * e1; t[0] = xi * e2; t[1] = xi * e2 * e3; }
        else { s[0] = xi * e2; s[1] = xi * e2 * e3; t[0] = xi; t[1] = xi * e1; }
    }
}

static double ss_jac(int rel, int reg, double xi, double e1, double e2) {
    if (rel == 3) return xi * xi * xi * e1 * e1 * e2;
    if (rel == 2) return xi * xi * xi * e1 * e1 * (reg == 0 ? 1.0 : e2);
    return xi * xi * xi * e2;
}

bool build_quadrature(Quadrature& q, int n_gauss) {
    if (!rule6(q.l1, q.l2, q.w)) return false;
    for (int i = 0; i < QP; i++) {
        q.lam[i][0] = 1 - q.l1[i] - q.l2[i];
        q.lam[i][1] = q.l1[i];
        q.lam[i][2] = q.l2[i];
    }
    q.ng = n_gauss;
    std::vector<double> gx, gw;
    gauss_legendre01(n_gauss, gx, gw);
    // near pairs (no common vertex): the collapsed Gauss-Legendre rule on each
    // triangle, s = (u, u v) with Jacobian u, in the reference parametrisation
    // of the singular tables
    {
        auto& tab = q.ss[0];
        tab.clear();
        for (int a = 0; a < n_gauss; a++)
            for (int b = 0; b < n_gauss; b++)
                for (int c = 0; c < n_gauss; c++)
                    for (int d = 0; d < n_gauss; d++) {
                        const double wt = gw[a] * gw[b] * gx[a] * gw[c] * gw[d] * gx[c];
                        tab.insert(tab.end(), {gx[a], gx[a] * gx[b], gx[c], gx[c] * gx[d], wt});
                    }
    }
    for (int rel = 1; rel <= 3; rel++) {
        int nreg = rel == 3 ? 6 : rel == 2 ? 5 : 2;
        auto& tab = q.ss[rel];
        tab.clear();
        for (int a = 0; a < n_gauss; a++)
            for (int b = 0; b < n_gauss; b++)
                for (int c = 0; c < n_gauss; c++)
                    for (int d = 0; d < n_gauss; d++)
                        for (int reg = 0; reg < nreg; reg++) {
                            double s[2], t[2];
                            ss_map(rel, reg, gx[a], gx[b], gx[c], gx[d], s, t);
                            double wt = gw[a] * gw[b] * gw[c] * gw[d] * ss_jac(rel, reg, gx[a], gx[b], gx[c]);
                            tab.insert(tab.end(), {s[0], s[1], t[0], t[1], wt});
                        }
    }
    return true;
}

// ---------------------------------------------------------------- geometry

static inline uint32_t spread10(uint32_t v) {
    v &= 1023u;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

std::string build_geometry(const std::vector<HostDomain>& doms, const Quadrature& q, Geometry& g) {
    g = Geometry();
    g.n_dom = (int)doms.size();
    if (g.n_dom == 0) return "no domain added";
    // ---- validation and offsets
    int64_t voff = 0, doff = 0;
    for (int d = 0; d < g.n_dom; d++) {
        const HostDomain& D = doms[d];
        if (D.nv < 3 || D.nt < 4) return "domain " + std::to_string(d) + ": too few vertices or triangles";
        std::unordered_map<uint64_t, int> edges;
        edges.reserve((size_t)D.nt * 3 * 2);
        for (int64_t t = 0; t < D.nt; t++) {
            const int32_t* v = &D.tris[3 * t];
            for (int i = 0; i < 3; i++)
                if (v[i] < 0 || v[i] >= D.nv) return "domain " + std::to_string(d) + ": triangle index out of range";
            if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2])
                return "domain " + std::to_string(d) + ": degenerate triangle";
            const double* a = &D.verts[3 * v[0]];
            const double* b = &D.verts[3 * v[1]];
            const double* c = &D.verts[3 * v[2]];
            double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
            double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
            double l = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            if (!(l > 0) || !std::isfinite(l)) return "domain " + std::to_string(d) + ": zero-area triangle";
            for (int i = 0; i < 3; i++) {
                uint64_t key = ((uint64_t)(uint32_t)v[i] << 32) | (uint32_t)v[(i + 1) % 3];
                if (++edges[key] > 1) return "domain " + std::to_string(d) + ": edge used twice in one direction (non-manifold or inconsistent orientation)";
            }
        }
        for (auto& kv : edges) {
            uint64_t rev = (kv.first << 32) | (kv.first >> 32);
            auto it = edges.find(rev);
            if (it == edges.end()) return "domain " + std::to_string(d) + ": open surface (boundary edge)";
        }
        g.dom_vert_off.push_back(voff);
        g.dom_dof_off.push_back(doff);
        g.dom_nv.push_back(D.nv);
        voff += D.nv;
        doff += 2 * D.nv;
    }
    g.n_vert = voff;
    g.n_dof = doff;
    g.v_dof1.resize(voff);
    g.v_dof2.resize(voff);
    for (int d = 0; d < g.n_dom; d++)
        for (int64_t v = 0; v < doms[d].nv; v++) {
            g.v_dof1[g.dom_vert_off[d] + v] = g.dom_dof_off[d] + v;
            g.v_dof2[g.dom_vert_off[d] + v] = g.dom_dof_off[d] + doms[d].nv + v;
        }
    // ---- tiling
    std::vector<std::vector<int>> order(g.n_dom);
    int tiles = 0;
    for (int d = 0; d < g.n_dom; d++) {
        const HostDomain& D = doms[d];
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        std::vector<double> cen(3 * D.nt);
        for (int64_t t = 0; t < D.nt; t++)
            for (int k = 0; k < 3; k++) {
                double c = (D.verts[3 * D.tris[3 * t] + k] + D.verts[3 * D.tris[3 * t + 1] + k] +
                            D.verts[3 * D.tris[3 * t + 2] + k]) / 3.0;
                cen[3 * t + k] = c;
                lo[k] = std::min(lo[k], c);
                hi[k] = std::max(hi[k], c);
            }
        double diag = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                (hi[2] - lo[2]) * (hi[2] - lo[2]));
        g.max_diameter = std::max(g.max_diameter, diag);
        double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
        std::vector<uint32_t> code(D.nt);
        for (int64_t t = 0; t < D.nt; t++) {
            uint32_t c[3];
            for (int k = 0; k < 3; k++) {
                double u = (cen[3 * t + k] - lo[k]) / ext;
                c[k] = (uint32_t)std::min(1023.0, std::max(0.0, u * 1023.0));
            }
            code[t] = spread10(c[0]) | (spread10(c[1]) << 1) | (spread10(c[2]) << 2);
        }
        order[d].resize(D.nt);
        std::iota(order[d].begin(), order[d].end(), 0);
        std::stable_sort(order[d].begin(), order[d].end(), [&](int a, int b) { return code[a] < code[b]; });
        g.dom_tile_begin.push_back(tiles);
        tiles += (int)((D.nt + TT - 1) / TT);
        g.dom_tile_end.push_back(tiles);
    }
    g.n_tiles = tiles;
    g.n_slots = (int64_t)tiles * TT;
    g.n_pts = (int64_t)tiles * TP;
    g.tile_c.assign(4 * (size_t)tiles, 0.0);
    g.tile_dom.assign(tiles, 0);
    g.tile_ntri.assign(tiles, 0);
    g.slot_v.assign(4 * g.n_slots, -1);
    g.slot_P.assign(9 * g.n_slots, 0.0);
    g.slot_n.assign(3 * g.n_slots, 0.0);
    g.slot_area.assign(g.n_slots, 0.0);
    g.slot_curl.assign(9 * g.n_slots, 0.0);
    g.slot_h.assign(g.n_slots, 0.0);
    g.pt_delta.assign(3 * g.n_pts, 0.0);
    g.pt_w.assign(g.n_pts, 0.0);
    std::vector<int64_t> slot_of_tri;  // per domain local triangle -> slot
    std::vector<std::vector<int64_t>> dom_slot(g.n_dom);
    std::vector<double> absP(3 * g.n_pts, 0.0);
    for (int d = 0; d < g.n_dom; d++) {
        const HostDomain& D = doms[d];
        dom_slot[d].assign(D.nt, -1);
        for (int64_t i = 0; i < D.nt; i++) {
            int tile = g.dom_tile_begin[d] + (int)(i / TT);
            int64_t slot = (int64_t)tile * TT + i % TT;
            int t = order[d][i];
            dom_slot[d][t] = slot;
            g.tile_dom[tile] = d;
            g.tile_ntri[tile]++;
            const int32_t* v = &D.tris[3 * t];
            const double* P[3] = {&D.verts[3 * v[0]], &D.verts[3 * v[1]], &D.verts[3 * v[2]]};
            for (int k = 0; k < 3; k++) g.slot_v[4 * slot + k] = (int)(g.dom_vert_off[d] + v[k]);
            g.slot_v[4 * slot + 3] = d;
            for (int k = 0; k < 3; k++)
                for (int c = 0; c < 3; c++) g.slot_P[9 * slot + 3 * k + c] = P[k][c];
            double e1[3], e2[3], cr[3];
            for (int c = 0; c < 3; c++) { e1[c] = P[1][c] - P[0][c]; e2[c] = P[2][c] - P[0][c]; }
            cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
            cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
            cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
            double l = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            double area = 0.5 * l;
            g.slot_area[slot] = area;
            for (int c = 0; c < 3; c++) g.slot_n[3 * slot + c] = cr[c] / l;
            // surface curl of hat function k: n x grad = (P_{k+1} - P_{k+2}) / (2|T|)
            for (int k = 0; k < 3; k++)
                for (int c = 0; c < 3; c++)
                    g.slot_curl[9 * slot + 3 * k + c] = (P[(k + 1) % 3][c] - P[(k + 2) % 3][c]) / (2.0 * area);
            for (int qi = 0; qi < QP; qi++) {
                int64_t p = slot * QP + qi;
                for (int c = 0; c < 3; c++)
                    absP[3 * p + c] = P[0][c] + q.l1[qi] * (P[1][c] - P[0][c]) + q.l2[qi] * (P[2][c] - P[0][c]);
                g.pt_w[p] = q.w[qi] * area;
            }
        }
    }
    for (int tile = 0; tile < tiles; tile++) {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        int nt = g.tile_ntri[tile];
        for (int64_t p = (int64_t)tile * TP; p < (int64_t)tile * TP + (int64_t)nt * QP; p++)
            for (int c = 0; c < 3; c++) { lo[c] = std::min(lo[c], absP[3 * p + c]); hi[c] = std::max(hi[c], absP[3 * p + c]); }
        double cc[3];
        for (int c = 0; c < 3; c++) cc[c] = 0.5 * (lo[c] + hi[c]);
        double rad = 0;
        for (int64_t p = (int64_t)tile * TP; p < (int64_t)tile * TP + (int64_t)nt * QP; p++) {
            double s = 0;
            for (int c = 0; c < 3; c++) {
                g.pt_delta[3 * p + c] = absP[3 * p + c] - cc[c];
                s += g.pt_delta[3 * p + c] * g.pt_delta[3 * p + c];
            }
            rad = std::max(rad, std::sqrt(s));
        }
        for (int c = 0; c < 3; c++) g.tile_c[4 * tile + c] = cc[c];
        g.tile_c[4 * tile + 3] = rad;
        for (int64_t slot = (int64_t)tile * TT; slot < (int64_t)tile * TT + nt; slot++) {
            double h = 0;
            for (int c = 0; c < 3; c++) h += g.slot_n[3 * slot + c] * (g.slot_P[9 * slot + c] - cc[c]);
            g.slot_h[slot] = h;
        }
    }
    // ---- vertex -> corner CSR
    g.vc_ptr.assign(g.n_vert + 1, 0);
    for (int64_t s = 0; s < g.n_slots; s++)
        if (g.slot_v[4 * s] >= 0)
            for (int k = 0; k < 3; k++) g.vc_ptr[g.slot_v[4 * s + k] + 1]++;
    for (int64_t v = 0; v < g.n_vert; v++) g.vc_ptr[v + 1] += g.vc_ptr[v];
    g.vc_idx.assign(g.vc_ptr[g.n_vert], 0);
    {
        std::vector<int64_t> fill(g.vc_ptr.begin(), g.vc_ptr.end() - 1);
        for (int64_t s = 0; s < g.n_slots; s++)
            if (g.slot_v[4 * s] >= 0)
                for (int k = 0; k < 3; k++) g.vc_idx[fill[g.slot_v[4 * s + k]]++] = (int32_t)(3 * s + k);
    }
    // ---- touching pairs (share at least one vertex), CSR over target slots
    std::vector<std::vector<std::pair<int32_t, int32_t>>> lists(g.n_slots);
    int64_t n_tri = 0;
    for (int d = 0; d < g.n_dom; d++) {
        const HostDomain& D = doms[d];
        n_tri += D.nt;
        std::vector<int64_t> vt_ptr(D.nv + 1, 0);
        for (int64_t t = 0; t < D.nt; t++)
            for (int k = 0; k < 3; k++) vt_ptr[D.tris[3 * t + k] + 1]++;
        for (int64_t v = 0; v < D.nv; v++) vt_ptr[v + 1] += vt_ptr[v];
        std::vector<int32_t> vt(vt_ptr[D.nv]);
        std::vector<int64_t> fill(vt_ptr.begin(), vt_ptr.end() - 1);
        for (int64_t t = 0; t < D.nt; t++)
            for (int k = 0; k < 3; k++) vt[fill[D.tris[3 * t + k]]++] = (int32_t)t;
        for (int64_t a = 0; a < D.nt; a++) {
            const int32_t* A = &D.tris[3 * a];
            std::vector<int32_t> cand;
            for (int k = 0; k < 3; k++)
                for (int64_t j = vt_ptr[A[k]]; j < vt_ptr[A[k] + 1]; j++) cand.push_back(vt[j]);
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            for (int32_t b : cand) {
                const int32_t* B = &D.tris[3 * b];
                int pa[3], pb[3], ns = 0, usedA[3] = {0, 0, 0}, usedB[3] = {0, 0, 0};
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++)
                        if (A[i] == B[j]) { pa[ns] = i; pb[ns] = j; usedA[i] = usedB[j] = 1; ns++; }
                int rel = ns;  // 1 vertex, 2 edge, 3 identical
                int ia = ns, ib = ns;
                for (int i = 0; i < 3; i++) { if (!usedA[i]) pa[ia++] = i; if (!usedB[i]) pb[ib++] = i; }
                int32_t code = rel | (pa[0] << 4) | (pa[1] << 6) | (pa[2] << 8) | (pb[0] << 10) | (pb[1] << 12) | (pb[2] << 14);
                lists[dom_slot[d][a]].push_back({(int32_t)dom_slot[d][b], code});
            }
        }
    }
    // ---- near pairs: no common vertex, centroids closer than twice the longer
    // of the two triangles' longest edges, within a domain or across domains.
    // The test is evaluated exactly as written (squared lengths, no fused
    // multiply-adds), so the library and an independent evaluation of the same
    // rule take the same decision.
    {
        struct Cen {
            double c[3], h2;
            int d;
            int32_t t;
        };
        std::vector<Cen> cs;
        cs.reserve((size_t)n_tri);
        double hmax2 = 0.0;
        for (int d = 0; d < g.n_dom; d++) {
            const HostDomain& D = doms[d];
            for (int64_t t = 0; t < D.nt; t++) {
                const double* P[3] = {&D.verts[3 * D.tris[3 * t]], &D.verts[3 * D.tris[3 * t + 1]],
                                      &D.verts[3 * D.tris[3 * t + 2]]};
                Cen e{};
                for (int k = 0; k < 3; k++) e.c[k] = (P[0][k] + P[1][k] + P[2][k]) / 3.0;
                for (int i = 0; i < 3; i++) {
                    const double* A = P[i];
                    const double* B = P[(i + 1) % 3];
                    const double x = B[0] - A[0], y = B[1] - A[1], z = B[2] - A[2];
                    const double l2 = x * x + y * y + z * z;
                    if (l2 > e.h2) e.h2 = l2;
                }
                e.d = d;
                e.t = (int32_t)t;
                hmax2 = std::max(hmax2, e.h2);
                cs.push_back(e);
            }
        }
        // uniform grid of cell 2 hmax: every near partner lies in the 27 neighbouring cells
        const double cell = 2.0 * std::sqrt(hmax2) * (1.0 + 1e-9);
        double lo[3] = {1e300, 1e300, 1e300};
        for (const Cen& e : cs)
            for (int k = 0; k < 3; k++) lo[k] = std::min(lo[k], e.c[k]);
        auto cell_of = [&](const double* c, int k) { return (int64_t)std::floor((c[k] - lo[k]) / cell); };
        auto key = [](int64_t i, int64_t j, int64_t k) { return (i * 1048576 + j) * 1048576 + k; };
        std::vector<std::pair<int64_t, int32_t>> keyed(cs.size());
        for (size_t i = 0; i < cs.size(); i++)
            keyed[i] = {key(cell_of(cs[i].c, 0), cell_of(cs[i].c, 1), cell_of(cs[i].c, 2)), (int32_t)i};
        std::sort(keyed.begin(), keyed.end());
        const int32_t near_code = 0 | (0 << 4) | (1 << 6) | (2 << 8) | (0 << 10) | (1 << 12) | (2 << 14);
        for (size_t ia = 0; ia < cs.size(); ia++) {
            const Cen& A = cs[ia];
            const int64_t ci = cell_of(A.c, 0), cj = cell_of(A.c, 1), ck = cell_of(A.c, 2);
            const int32_t* TA = &doms[A.d].tris[3 * (int64_t)A.t];
            for (int64_t di = -1; di <= 1; di++)
                for (int64_t dj = -1; dj <= 1; dj++)
                    for (int64_t dk = -1; dk <= 1; dk++) {
                        const int64_t kk = key(ci + di, cj + dj, ck + dk);
                        auto it = std::lower_bound(keyed.begin(), keyed.end(), std::make_pair(kk, (int32_t)INT32_MIN));
                        for (; it != keyed.end() && it->first == kk; ++it) {
                            const Cen& B = cs[it->second];
                            if (it->second == (int32_t)ia) continue;
                            if (B.d == A.d) {  // touching pairs have their own rules
                                const int32_t* TB = &doms[B.d].tris[3 * (int64_t)B.t];
                                bool share = false;
                                for (int u = 0; u < 3; u++)
                                    for (int v = 0; v < 3; v++) share |= TA[u] == TB[v];
                                if (share) continue;
                            }
                            const double x = A.c[0] - B.c[0], y = A.c[1] - B.c[1], z = A.c[2] - B.c[2];
                            const double h2 = std::max(A.h2, B.h2);
                            if (x * x + y * y + z * z < 4.0 * h2)
                                lists[dom_slot[A.d][A.t]].push_back({(int32_t)dom_slot[B.d][B.t], near_code});
                        }
                    }
        }
    }
    g.n_tri = n_tri;
    g.np_ptr.assign(g.n_slots + 1, 0);
    for (int64_t s = 0; s < g.n_slots; s++) g.np_ptr[s + 1] = g.np_ptr[s] + (int64_t)lists[s].size();
    g.np_src.resize(g.np_ptr[g.n_slots]);
    g.np_code.resize(g.np_ptr[g.n_slots]);
    for (int64_t s = 0; s < g.n_slots; s++)
        for (size_t i = 0; i < lists[s].size(); i++) {
            g.np_src[g.np_ptr[s] + i] = lists[s][i].first;
            g.np_code[g.np_ptr[s] + i] = lists[s][i].second;
        }
    return "";
}

}  // namespace gbem
