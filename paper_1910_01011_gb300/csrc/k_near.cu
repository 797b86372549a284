// k_near.cu -- near-field correction for touching and near triangle pairs (FP64).
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
    near_build_kernel<<<dim3((unsigned)a.n_pairs, a.n_slot_k), NEAR_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_near_combine(const NearCombineArgs& a, cudaStream_t s) {
    if (a.n_pairs <= 0) return cudaSuccess;
    near_combine_kernel<<<(unsigned)((a.n_pairs + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gbem
