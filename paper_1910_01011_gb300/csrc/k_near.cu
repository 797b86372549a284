// k_near.cu -- near-field correction for touching and near triangle pairs
// (FP64, or FP64-accurate double-float point evaluations by default).
//
// For every pair of triangles of one surface that shares a vertex, an edge
// or is identical, the far-field kernel's regular 6-point x 6-point rule is
// wrong (or, for the identical pair, skipped).  This file integrates the
// pair with the Sauter-Schwab regularising maps (Sauter & Schwab, Boundary
// Element Methods, Sec. 5.2; the paper leaves quadrature to its BEM library,
// Sec. 3).  Pairs without a common vertex whose centroids are closer than
// twice the longer of their longest edges (within a surface or across
// domains) are integrated with a collapsed Gauss-Legendre rule on each
// triangle (table 0).  Either way the kernel subtracts exactly what the
// far-field kernel adds, giving
// per-pair 3x3 corrections of V, K, K' (paper App. A); W follows from V by
// its integration-by-parts form: W_ab = curl_a.curl_b sum(V) - k^2 (n_x.n_y) V_ab.
// The corrections of both wavenumbers of a domain are combined with the
// block coefficients of the PMCHWT system (Sec. 2.2) into four 3x3 blocks
// (row1<-psi, row1<-phi, row2<-psi, row2<-phi), applied per matvec by the
// projection kernel.
#include "df_math.cuh"
#include "internal.h"

namespace gbem {

constexpr int NEAR_THREADS = 128;
constexpr int NACC = 27;  // V, K, K' (3x3 complex each)

__device__ __forceinline__ void kernel_eval(const double* x, const double* y, const double* nx, const double* ny,
                                            double kr, double ki, double w, const double* lx, const double* ly,
                                            double (*acc)[2]) {
    const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const double rinv = 1.0 / r;
    double sn, cs;
    sincos(kr * r, &sn, &cs);
    const double a = exp(-ki * r) * rinv * 0.07957747154594767 * w;  // w G magnitude
    const double Gr = a * cs, Gi = a * sn;
    const double u = -ki - rinv;                                   // Re(ik - 1/r)
    const double Fr = (Gr * u - Gi * kr) * rinv, Fi = (Gr * kr + Gi * u) * rinv;
    const double dny = -(d0 * ny[0] + d1 * ny[1] + d2 * ny[2]);    // (y - x).n_y
    const double dnx = d0 * nx[0] + d1 * nx[1] + d2 * nx[2];       // (x - y).n_x
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            const double pp = lx[i] * ly[j];
            acc[3 * i + j][0] += Gr * pp;
            acc[3 * i + j][1] += Gi * pp;
            acc[9 + 3 * i + j][0] += Fr * dny * pp;
            acc[9 + 3 * i + j][1] += Fi * dny * pp;
            acc[18 + 3 * i + j][0] += Fr * dnx * pp;
            acc[18 + 3 * i + j][1] += Fi * dnx * pp;
        }
}

// grid: (pair, wavenumber slot); one CTA integrates one pair at one k.
__global__ void __launch_bounds__(NEAR_THREADS) near_build_kernel(NearArgs A) {
    const int64_t pi = blockIdx.x;
    const int sl = blockIdx.y;
    const int tgt = A.pair_tgt[pi], src = A.pair_src[pi];
    const int code = A.pair_code[pi];
    const int rel = code & 15;
    int pa[3], pb[3];
    for (int i = 0; i < 3; i++) {
        pa[i] = (code >> (4 + 2 * i)) & 3;
        pb[i] = (code >> (10 + 2 * i)) & 3;
    }
    const int dom = A.slot_dom[4 * tgt + 3];
    const double2 k = sl == 0 ? A.k[0] : A.kdom[dom];
    // the own-domain wavenumber applies only to pairs within the target's domain
    const bool live = sl == 0 || A.slot_dom[4 * src + 3] == dom;
    // reordered vertices: shared ones first, in matching order
    double PX[3][3], PY[3][3], OX[3][3], OY[3][3], nx[3], ny[3];
    for (int i = 0; i < 3; i++)
        for (int c = 0; c < 3; c++) {
            PX[i][c] = A.slot_P[(int64_t)tgt * 9 + 3 * pa[i] + c];
            PY[i][c] = A.slot_P[(int64_t)src * 9 + 3 * pb[i] + c];
            OX[i][c] = A.slot_P[(int64_t)tgt * 9 + 3 * i + c];
            OY[i][c] = A.slot_P[(int64_t)src * 9 + 3 * i + c];
        }
    for (int c = 0; c < 3; c++) {
        nx[c] = A.slot_n[(int64_t)tgt * 3 + c];
        ny[c] = A.slot_n[(int64_t)src * 3 + c];
    }
    const double ax = A.slot_area[tgt], ay = A.slot_area[src];
    double acc[NACC][2];
    for (int i = 0; i < NACC; i++) acc[i][0] = acc[i][1] = 0.0;
    // Sauter-Schwab part, accumulated in the ORIGINAL local order
    const double* tab = A.ss_tab[rel];
    const int n = live ? A.ss_n[rel] : 0;
    const double scale = 4.0 * ax * ay;
    for (int idx = threadIdx.x; idx < n; idx += NEAR_THREADS) {
        const double s1 = tab[5 * idx], s2 = tab[5 * idx + 1], t1 = tab[5 * idx + 2], t2 = tab[5 * idx + 3];
        const double w = tab[5 * idx + 4] * scale;
        double x[3], y[3], lxr[3] = {1 - s1, s1 - s2, s2}, lyr[3] = {1 - t1, t1 - t2, t2}, lx[3], ly[3];
        for (int c = 0; c < 3; c++) {
            x[c] = PX[0][c] + s1 * (PX[1][c] - PX[0][c]) + s2 * (PX[2][c] - PX[1][c]);
            y[c] = PY[0][c] + t1 * (PY[1][c] - PY[0][c]) + t2 * (PY[2][c] - PY[1][c]);
        }
        for (int i = 0; i < 3; i++) {
            lx[pa[i]] = lxr[i];
            ly[pb[i]] = lyr[i];
        }
        kernel_eval(x, y, nx, ny, k.x, k.y, w, lx, ly, acc);
    }
    // minus the regular rule the far-field kernel applied (not for identical pairs)
    if (rel != 3 && live) {
        for (int idx = threadIdx.x; idx < QP * QP; idx += NEAR_THREADS) {
            const int qa = idx / QP, qb = idx % QP;
            const double l1 = A.rule[3 * qa], l2 = A.rule[3 * qa + 1], wa = A.rule[3 * qa + 2];
            const double m1 = A.rule[3 * qb], m2 = A.rule[3 * qb + 1], wb = A.rule[3 * qb + 2];
            double x[3], y[3];
            for (int c = 0; c < 3; c++) {
                x[c] = OX[0][c] + l1 * (OX[1][c] - OX[0][c]) + l2 * (OX[2][c] - OX[0][c]);
                y[c] = OY[0][c] + m1 * (OY[1][c] - OY[0][c]) + m2 * (OY[2][c] - OY[0][c]);
            }
            const double lx[3] = {1 - l1 - l2, l1, l2}, ly[3] = {1 - m1 - m2, m1, m2};
            kernel_eval(x, y, nx, ny, k.x, k.y, -wa * wb * ax * ay, lx, ly, acc);
        }
    }
    // block reduction
    __shared__ double red[NEAR_THREADS / 32][NACC][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < NACC; i++)
        for (int c = 0; c < 2; c++) {
            double v = acc[i][c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][i][c] = v;
        }
    __syncthreads();
    if (threadIdx.x < NACC * 2) {
        const int i = threadIdx.x >> 1, c = threadIdx.x & 1;
        double v = 0;
        for (int w = 0; w < NEAR_THREADS / 32; w++) v += red[w][i][c];
        double* out = reinterpret_cast<double*>(A.raw + ((int64_t)pi * A.n_slot_k + sl) * NACC);
        out[2 * i + c] = v;
    }
}

// ---- the same integrals with double-float point evaluations (df_math.cuh):
// GB300 runs FP64 at ~1/64 of its FP32 rate and every point pair costs a
// square root, a reciprocal and a sincos; the pair's geometry is split once
// into shared memory, the table points are read as (hi, lo) floats, and the
// 27 complex moments of each thread are converted to FP64 once for the
// block reduction (relative accuracy ~1e-13).

struct NearGeomDF {
    dfl X0[3], X1[3], X2[3], Y0[3], Y1[3], Y2[3];  // Sauter-Schwab parametrisations (reordered vertices)
    dfl O0[3], Ou[3], Ov[3], Q0[3], Qu[3], Qv[3];  // regular-rule parametrisations (original order)
    dfl nx[3], ny[3], scale, axay;
};

__device__ __forceinline__ dfl split_d(double v) {
    const float h = (float)v;
    return dfl{h, (float)(v - (double)h)};
}

template <bool ATTEN>
__device__ __forceinline__ void kernel_eval_df(const dfl (&x)[3], const dfl (&y)[3], const NearGeomDF& G, dfl kr,
                                               dfl ki, dfl w, const dfl (&lx)[3], const dfl (&ly)[3],
                                               const NearArgs& A, const float4* __restrict__ tab,
                                               const float2* __restrict__ etab, dfl (&acc)[NACC][2]) {
    const dfl d0 = dsub(x[0], y[0]), d1 = dsub(x[1], y[1]), d2 = dsub(x[2], y[2]);
    dfl r, ri;
    dsqrt_rinv(dadd(dadd(dsqr(d0), dsqr(d1)), dsqr(d2)), r, ri);
    dfl sn, cs;
    dsincos(dmul(kr, r), A.c, tab, sn, cs);
    dfl a = dmul(dmul(ri, dfl{A.i4h, A.i4l}), w);  // w G magnitude
    if (ATTEN) a = dmul(a, dexp_neg(dmul(ki, r), A.c, etab));
    const dfl Gr = dmul(a, cs), Gi = dmul(a, sn);
    const dfl u = dsub(dneg(ki), ri);  // Re(ik - 1/r)
    const dfl Fr = dmul(dsub(dmul(Gr, u), dmul(Gi, kr)), ri);
    const dfl Fi = dmul(dadd(dmul(Gr, kr), dmul(Gi, u)), ri);
    const dfl dny = dneg(dadd(dadd(dmul(d0, G.ny[0]), dmul(d1, G.ny[1])), dmul(d2, G.ny[2])));  // (y - x).n_y
    const dfl dnx = dadd(dadd(dmul(d0, G.nx[0]), dmul(d1, G.nx[1])), dmul(d2, G.nx[2]));        // (x - y).n_x
    const dfl Fyr = dmul(Fr, dny), Fyi = dmul(Fi, dny), Fxr = dmul(Fr, dnx), Fxi = dmul(Fi, dnx);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const dfl pp = dmul(lx[i], ly[j]);
            dmac(acc[3 * i + j][0], Gr, pp, 1.0f);
            dmac(acc[3 * i + j][1], Gi, pp, 1.0f);
            dmac(acc[9 + 3 * i + j][0], Fyr, pp, 1.0f);
            dmac(acc[9 + 3 * i + j][1], Fyi, pp, 1.0f);
            dmac(acc[18 + 3 * i + j][0], Fxr, pp, 1.0f);
            dmac(acc[18 + 3 * i + j][1], Fxi, pp, 1.0f);
        }
}

// lx[pa[i]] = v[i] for a permutation pa, without run-time register indexing
__device__ __forceinline__ void permute3(const dfl (&v)[3], const int (&pa)[3], dfl (&out)[3]) {
#pragma unroll
    for (int j = 0; j < 3; j++) out[j] = pa[0] == j ? v[0] : pa[1] == j ? v[1] : v[2];
}

template <bool ATTEN>
__device__ __forceinline__ void near_df_body(const NearArgs& A, const NearGeomDF& G, int rel, const int (&pa)[3],
                                             const int (&pb)[3], dfl kr, dfl ki, bool live,
                                             const float4* __restrict__ tab, const float2* __restrict__ etab,
                                             dfl (&acc)[NACC][2]) {
    const int n = live ? A.ss_n[rel] : 0;
    const float* th = A.ss_tabf[rel];
    const float* tl = th + 5 * (int64_t)A.ss_n[rel];
    for (int idx = threadIdx.x; idx < n; idx += NEAR_THREADS) {
        const dfl s1 = {th[5 * idx], tl[5 * idx]}, s2 = {th[5 * idx + 1], tl[5 * idx + 1]};
        const dfl t1 = {th[5 * idx + 2], tl[5 * idx + 2]}, t2 = {th[5 * idx + 3], tl[5 * idx + 3]};
        const dfl w = dmul(dfl{th[5 * idx + 4], tl[5 * idx + 4]}, G.scale);
        dfl x[3], y[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            x[c] = dadd(dadd(G.X0[c], dmul(s1, G.X1[c])), dmul(s2, G.X2[c]));
            y[c] = dadd(dadd(G.Y0[c], dmul(t1, G.Y1[c])), dmul(t2, G.Y2[c]));
        }
        const dfl lxr[3] = {dsub(dfl{1.0f, 0.0f}, s1), dsub(s1, s2), s2};
        const dfl lyr[3] = {dsub(dfl{1.0f, 0.0f}, t1), dsub(t1, t2), t2};
        dfl lx[3], ly[3];
        permute3(lxr, pa, lx);
        permute3(lyr, pb, ly);
        kernel_eval_df<ATTEN>(x, y, G, kr, ki, w, lx, ly, A, tab, etab, acc);
    }
    // minus the regular rule the far-field kernel applied (not for identical pairs)
    if (rel != 3 && live)
        for (int idx = threadIdx.x; idx < QP * QP; idx += NEAR_THREADS) {
            const int qa = idx / QP, qb = idx % QP;
            const dfl l1 = {A.rule_h[3 * qa], A.rule_l[3 * qa]}, l2 = {A.rule_h[3 * qa + 1], A.rule_l[3 * qa + 1]};
            const dfl wa = {A.rule_h[3 * qa + 2], A.rule_l[3 * qa + 2]};
            const dfl m1 = {A.rule_h[3 * qb], A.rule_l[3 * qb]}, m2 = {A.rule_h[3 * qb + 1], A.rule_l[3 * qb + 1]};
            const dfl wb = {A.rule_h[3 * qb + 2], A.rule_l[3 * qb + 2]};
            dfl x[3], y[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                x[c] = dadd(dadd(G.O0[c], dmul(l1, G.Ou[c])), dmul(l2, G.Ov[c]));
                y[c] = dadd(dadd(G.Q0[c], dmul(m1, G.Qu[c])), dmul(m2, G.Qv[c]));
            }
            const dfl lx[3] = {dsub(dsub(dfl{1.0f, 0.0f}, l1), l2), l1, l2};
            const dfl ly[3] = {dsub(dsub(dfl{1.0f, 0.0f}, m1), m2), m1, m2};
            kernel_eval_df<ATTEN>(x, y, G, kr, ki, dneg(dmul(dmul(wa, wb), G.axay)), lx, ly, A, tab, etab, acc);
        }
}

// grid: (pair, wavenumber slot); one CTA integrates one pair at one k.
__global__ void __launch_bounds__(NEAR_THREADS) near_build_df_kernel(NearArgs A) {
    __shared__ float4 tab[128];
    __shared__ float2 etab[64];
    __shared__ NearGeomDF G;
    const int64_t pi = blockIdx.x;
    const int sl = blockIdx.y;
    const int tgt = A.pair_tgt[pi], src = A.pair_src[pi];
    const int code = A.pair_code[pi];
    const int rel = code & 15;
    int pa[3], pb[3];
    for (int i = 0; i < 3; i++) {
        pa[i] = (code >> (4 + 2 * i)) & 3;
        pb[i] = (code >> (10 + 2 * i)) & 3;
    }
    const int dom = A.slot_dom[4 * tgt + 3];
    const float4 kk = sl == 0 ? A.k0df : A.kdf[dom];
    const dfl kr = {kk.x, kk.y}, ki = {kk.z, kk.w};
    const bool live = sl == 0 || A.slot_dom[4 * src + 3] == dom;
    for (int i = threadIdx.x; i < 128; i += NEAR_THREADS) tab[i] = A.sctab[i];
    for (int i = threadIdx.x; i < 64; i += NEAR_THREADS) etab[i] = A.extab[i];
    if (threadIdx.x == 0) {
        // the pair's geometry in FP64, differences formed before the split
        const double* P = A.slot_P;
        for (int c = 0; c < 3; c++) {
            const double px[3] = {P[(int64_t)tgt * 9 + 3 * pa[0] + c], P[(int64_t)tgt * 9 + 3 * pa[1] + c],
                                  P[(int64_t)tgt * 9 + 3 * pa[2] + c]};
            const double py[3] = {P[(int64_t)src * 9 + 3 * pb[0] + c], P[(int64_t)src * 9 + 3 * pb[1] + c],
                                  P[(int64_t)src * 9 + 3 * pb[2] + c]};
            const double ox[3] = {P[(int64_t)tgt * 9 + c], P[(int64_t)tgt * 9 + 3 + c], P[(int64_t)tgt * 9 + 6 + c]};
            const double oy[3] = {P[(int64_t)src * 9 + c], P[(int64_t)src * 9 + 3 + c], P[(int64_t)src * 9 + 6 + c]};
            G.X0[c] = split_d(px[0]);
            G.X1[c] = split_d(px[1] - px[0]);
            G.X2[c] = split_d(px[2] - px[1]);
            G.Y0[c] = split_d(py[0]);
            G.Y1[c] = split_d(py[1] - py[0]);
            G.Y2[c] = split_d(py[2] - py[1]);
            G.O0[c] = split_d(ox[0]);
            G.Ou[c] = split_d(ox[1] - ox[0]);
            G.Ov[c] = split_d(ox[2] - ox[0]);
            G.Q0[c] = split_d(oy[0]);
            G.Qu[c] = split_d(oy[1] - oy[0]);
            G.Qv[c] = split_d(oy[2] - oy[0]);
            G.nx[c] = split_d(A.slot_n[(int64_t)tgt * 3 + c]);
            G.ny[c] = split_d(A.slot_n[(int64_t)src * 3 + c]);
        }
        const double ax = A.slot_area[tgt], ay = A.slot_area[src];
        G.scale = split_d(4.0 * ax * ay);
        G.axay = split_d(ax * ay);
    }
    __syncthreads();
    dfl acc[NACC][2];
#pragma unroll
    for (int i = 0; i < NACC; i++) acc[i][0] = acc[i][1] = dfl{0.0f, 0.0f};
    if (kk.z != 0.0f || kk.w != 0.0f) near_df_body<true>(A, G, rel, pa, pb, kr, ki, live, tab, etab, acc);
    else near_df_body<false>(A, G, rel, pa, pb, kr, ki, live, tab, etab, acc);
    // block reduction in FP64: it runs on the FP64 pipe beside the FP32 point
    // evaluations of the other warps (a double-float shuffle reduction was
    // measured slower: 394 against 307 ms on the 8k-triangle rib scene, the
    // FP32 pipe being the busier one at eight warps per SM)
    __shared__ double red[NEAR_THREADS / 32][NACC][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NACC; i++)
#pragma unroll
        for (int c = 0; c < 2; c++) {
            double v = (double)acc[i][c].h + (double)acc[i][c].l;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][i][c] = v;
        }
    __syncthreads();
    if (threadIdx.x < NACC * 2) {
        const int i = threadIdx.x >> 1, c = threadIdx.x & 1;
        double v = 0;
        for (int w = 0; w < NEAR_THREADS / 32; w++) v += red[w][i][c];
        double* out = reinterpret_cast<double*>(A.raw + ((int64_t)pi * A.n_slot_k + sl) * NACC);
        out[2 * i + c] = v;
    }
}

__global__ void near_combine_kernel(NearCombineArgs A) {
    const int64_t pi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= A.n_pairs) return;
    const int tgt = A.pair_tgt[pi], src = A.pair_src[pi];
    const int dom = A.slot_v[tgt].w;
    double cc[3][3], nn = 0;
    for (int c = 0; c < 3; c++) nn += A.slot_n[(int64_t)tgt * 3 + c] * A.slot_n[(int64_t)src * 3 + c];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int c = 0; c < 3; c++)
                s += A.slot_curl[(int64_t)tgt * 9 + 3 * i + c] * A.slot_curl[(int64_t)src * 9 + 3 * j + c];
            cc[i][j] = s;
        }
    double B[4][9][2];
    for (int b = 0; b < 4; b++)
        for (int e = 0; e < 9; e++) B[b][e][0] = B[b][e][1] = 0.0;
    for (int sl = 0; sl < A.n_slot_k; sl++) {
        const SlotCoef cf = A.coef[dom * 2 + sl];
        const double2* R = A.raw + (pi * A.n_slot_k + sl) * NACC;
        double ig_r = 0, ig_i = 0;
        for (int e = 0; e < 9; e++) {
            ig_r += R[e].x;
            ig_i += R[e].y;
        }
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                const int e = 3 * i + j;
                const double2 V = R[e], K = R[9 + e], Kp = R[18 + e];
                // W = curl.curl * sum(V) - k^2 (n_x.n_y) V
                const double kvr = cf.k2re * V.x - cf.k2im * V.y, kvi = cf.k2re * V.y + cf.k2im * V.x;
                const double Wr = cc[i][j] * ig_r - nn * kvr, Wi = cc[i][j] * ig_i - nn * kvi;
                B[0][e][0] += cf.cV * V.x;
                B[0][e][1] += cf.cV * V.y;
                B[1][e][0] -= cf.cK * K.x;
                B[1][e][1] -= cf.cK * K.y;
                B[2][e][0] += cf.cKp * Kp.x;
                B[2][e][1] += cf.cKp * Kp.y;
                B[3][e][0] += cf.cW * Wr;
                B[3][e][1] += cf.cW * Wi;
            }
    }
    for (int b = 0; b < 4; b++)
        for (int e = 0; e < 9; e++) {
            A.nb64[(pi * 4 + b) * 9 + e] = make_double2(B[b][e][0], B[b][e][1]);
            A.nb32[(pi * 4 + b) * 9 + e] = make_float2((float)B[b][e][0], (float)B[b][e][1]);
        }
}

cudaError_t launch_near_build(const NearArgs& a, cudaStream_t s) {
    if (a.n_pairs <= 0) return cudaSuccess;
    // one launch per <= 65535 pairs is not needed: grid.x may be up to 2^31-1
    if (a.use_df) near_build_df_kernel<<<dim3((unsigned)a.n_pairs, a.n_slot_k), NEAR_THREADS, 0, s>>>(a);
    else near_build_kernel<<<dim3((unsigned)a.n_pairs, a.n_slot_k), NEAR_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_near_combine(const NearCombineArgs& a, cudaStream_t s) {
    if (a.n_pairs <= 0) return cudaSuccess;
    near_combine_kernel<<<(unsigned)((a.n_pairs + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gbem
