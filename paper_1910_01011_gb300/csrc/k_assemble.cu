// k_assemble.cu -- dense assembly of the PMCHWT Galerkin matrix A_hat
// (paper Sec. 2.2-2.3) in complex64, for the multi-right-hand-side path
// that applies it with the tensor-core GEMM (k_gemm.cu).
//
// Entry (row r, column q) of A_hat collects, over test triangles tau with
// vertex a = r and trial triangles t with vertex b = q, the 3x3 local
// Galerkin matrices of V, K, K' (regular 6-point rule on both triangles,
// FP32 with the tile-local phase of the far-field kernel) combined with the
// block coefficients of the system:
//   row1<-psi: cV V,  row1<-phi: -cK K,  row2<-psi: cKp K',
//   row2<-phi: cW (curl_a.curl_b sum(V) - k^2 n_x.n_y V)   (W by parts).
// Identical pairs are skipped here; every touching pair then receives its
// Sauter-Schwab correction block (k_near.cu).  Local blocks are added into
// the matrix with FP32 atomics (set-up only; the order of additions varies
// between runs at the level of FP32 rounding).
#include <cuda_runtime.h>

#include <cstdint>

#include "ctx.h"
#include "df_math.cuh"
#include "internal.h"

namespace gbem {

struct AssembleArgs {
    const float4* pg;       // points (dx, dy, dz, w)
    const float4* tg;       // triangles (n, h)
    const double4* tc;      // tile centres
    const int* tntri;
    const int4* slot_v;
    const double* slot_curl;
    const int64_t* v_dof1;
    const int64_t* v_dof2;
    const SlotCoef* coef;   // [n_dom*2]
    const int2* dom_tiles;
    const double2* kdom;
    double2 k0;
    int slot;               // 0: exterior k0 on all pairs; 1: own-domain k_j on own-domain pairs
    int n_tiles;
    int chunk_tiles;
    int64_t n;              // matrix dimension (leading dimension)
    float2* A;              // dense, row-major, n x n
    float lam[QP][3];
    double lam64[QP][3];
};

__device__ __forceinline__ float a_reduce_phase(double t) {
    const double two_pi_hi = 6.283185307179586, two_pi_lo = 2.4492935982947064e-16;
    double nn = rint(t * 0.15915494309189535);
    double r = fma(-nn, two_pi_hi, t);
    r = fma(-nn, two_pi_lo, r);
    return (float)r;
}

// grid (target tile, source chunk); thread = target triangle of the tile.
__global__ void __launch_bounds__(TT) assemble_kernel(AssembleArgs a) {
    const int tt = blockIdx.x;
    const int tl = threadIdx.x;
    const int64_t ts = (int64_t)tt * TT + tl;
    const int4 tv = a.slot_v[ts];
    if (tv.x < 0) return;
    const int dom = tv.w;
    const int2 dr = a.dom_tiles[dom];
    int sb = blockIdx.y * a.chunk_tiles, se = min(sb + a.chunk_tiles, a.n_tiles);
    if (a.slot == 1) {  // interior wavenumber: own-domain sources only
        sb = max(sb, dr.x);
        se = min(se, dr.y);
    }
    if (sb >= se) return;
    const double2 kd = a.slot == 0 ? a.k0 : a.kdom[dom];
    const float kr = (float)kd.x, nki = (float)-kd.y, nkil2 = (float)(-kd.y * 1.4426950408889634);
    const SlotCoef cf = a.coef[dom * 2 + a.slot];
    const float inv4pi = 0.0795774715459476678f;
    const float4 ng = a.tg[ts];
    float4 xs[QP];
    for (int q = 0; q < QP; q++) xs[q] = a.pg[ts * QP + q];
    float cx[3][3];
    for (int i = 0; i < 3; i++)
        for (int c = 0; c < 3; c++) cx[i][c] = (float)a.slot_curl[ts * 9 + 3 * i + c];
    const double4 ct = a.tc[tt];
    const int64_t ra[3] = {a.v_dof1[tv.x], a.v_dof1[tv.y], a.v_dof1[tv.z]};
    const int64_t rb[3] = {a.v_dof2[tv.x], a.v_dof2[tv.y], a.v_dof2[tv.z]};
    for (int s = sb; s < se; s++) {
        const double4 cs = a.tc[s];
        const double Dx = ct.x - cs.x, Dy = ct.y - cs.y, Dz = ct.z - cs.z;
        const double R = sqrt(Dx * Dx + Dy * Dy + Dz * Dz);
        const float D2x = (float)(2 * Dx), D2y = (float)(2 * Dy), D2z = (float)(2 * Dz), Rc2 = (float)(R * R);
        const float Rc = (float)R, th = a_reduce_phase(kd.x * R);
        const float nD = 0.5f * (ng.x * D2x + ng.y * D2y + ng.z * D2z);
        const int ntri = a.tntri[s];
        for (int sl = 0; sl < ntri; sl++) {
            const int64_t ss = (int64_t)s * TT + sl;
            if (ss == ts) continue;  // identical pair: near-field block only
            const float4 sg = a.tg[ss];
            float V[3][3][2] = {}, K[3][3][2] = {}, Kp[3][3][2] = {};
            for (int qx = 0; qx < QP; qx++) {
                const float4 x = xs[qx];
                const float Xx = x.x + 0.5f * D2x, Xy = x.y + 0.5f * D2y, Xz = x.z + 0.5f * D2z;
                const float fK = sg.w - (sg.x * Xx + sg.y * Xy + sg.z * Xz);   // n_t.(y - x)
                float hV[3][2] = {}, hK[3][2] = {}, hKp[3][2] = {};
                for (int qy = 0; qy < QP; qy++) {
                    const float4 y = a.pg[ss * QP + qy];
                    const float ex = x.x - y.x, ey = x.y - y.y, ez = x.z - y.z;
                    const float sd = ex * (D2x + ex) + ey * (D2y + ey) + ez * (D2z + ez);
                    const float r2 = Rc2 + sd;
                    const float rinv = rsqrtf(r2);
                    const float r = r2 * rinv;
                    const float rho = __fdividef(sd, r + Rc);
                    float sn, cs2;
                    __sincosf(fmaf(kr, rho, th), &sn, &cs2);
                    const float am = (nki != 0.f ? exp2f(nkil2 * r) : 1.f) * rinv;
                    const float Gr = am * cs2, Gi = am * sn;
                    const float u = nki - rinv;
                    const float Fr = (Gr * u - Gi * kr) * rinv, Fi = (Gr * kr + Gi * u) * rinv;
                    const float ndot = ng.x * ex + ng.y * ey + ng.z * ez + nD;    // n_x.(x - y)
                    for (int b = 0; b < 3; b++) {
                        const float wl = y.w * a.lam[qy][b];
                        hV[b][0] = fmaf(wl, Gr, hV[b][0]);
                        hV[b][1] = fmaf(wl, Gi, hV[b][1]);
                        hK[b][0] = fmaf(wl, Fr, hK[b][0]);
                        hK[b][1] = fmaf(wl, Fi, hK[b][1]);
                        hKp[b][0] = fmaf(wl * ndot, Fr, hKp[b][0]);
                        hKp[b][1] = fmaf(wl * ndot, Fi, hKp[b][1]);
                    }
                }
                for (int i = 0; i < 3; i++) {
                    const float wx = x.w * a.lam[qx][i] * inv4pi;
                    for (int b = 0; b < 3; b++) {
                        V[i][b][0] = fmaf(wx, hV[b][0], V[i][b][0]);
                        V[i][b][1] = fmaf(wx, hV[b][1], V[i][b][1]);
                        K[i][b][0] = fmaf(wx * fK, hK[b][0], K[i][b][0]);
                        K[i][b][1] = fmaf(wx * fK, hK[b][1], K[i][b][1]);
                        Kp[i][b][0] = fmaf(wx, hKp[b][0], Kp[i][b][0]);
                        Kp[i][b][1] = fmaf(wx, hKp[b][1], Kp[i][b][1]);
                    }
                }
            }
            // W by parts, then the four system blocks
            float sr = 0, si = 0;
            for (int i = 0; i < 3; i++)
                for (int b = 0; b < 3; b++) {
                    sr += V[i][b][0];
                    si += V[i][b][1];
                }
            const float nn = ng.x * sg.x + ng.y * sg.y + ng.z * sg.z;
            const int4 sv = a.slot_v[ss];
            const int vb[3] = {sv.x, sv.y, sv.z};
            for (int b = 0; b < 3; b++) {
                const int64_t ca = a.v_dof1[vb[b]], cb = a.v_dof2[vb[b]];
                const float cyx = (float)a.slot_curl[ss * 9 + 3 * b], cyy = (float)a.slot_curl[ss * 9 + 3 * b + 1],
                            cyz = (float)a.slot_curl[ss * 9 + 3 * b + 2];
                for (int i = 0; i < 3; i++) {
                    const float cc = cx[i][0] * cyx + cx[i][1] * cyy + cx[i][2] * cyz;
                    const float kvr = (float)cf.k2re * V[i][b][0] - (float)cf.k2im * V[i][b][1];
                    const float kvi = (float)cf.k2re * V[i][b][1] + (float)cf.k2im * V[i][b][0];
                    const float Wr = cc * sr - nn * kvr, Wi = cc * si - nn * kvi;
                    atomicAdd(&a.A[ra[i] * a.n + ca], make_float2((float)cf.cV * V[i][b][0], (float)cf.cV * V[i][b][1]));
                    atomicAdd(&a.A[ra[i] * a.n + cb], make_float2(-(float)cf.cK * K[i][b][0], -(float)cf.cK * K[i][b][1]));
                    atomicAdd(&a.A[rb[i] * a.n + ca], make_float2((float)cf.cKp * Kp[i][b][0], (float)cf.cKp * Kp[i][b][1]));
                    atomicAdd(&a.A[rb[i] * a.n + cb], make_float2((float)cf.cW * Wr, (float)cf.cW * Wi));
                }
            }
        }
    }
}

// FP64 version of the assembly (straight FP64 distances and transcendentals),
// for the refinement residual: entries accumulated with FP64 atomics.
__global__ void __launch_bounds__(TT) assemble64_kernel(AssembleArgs a, const double4* pg64, const double4* tg64,
                                                        double2* A64) {
    const int tt = blockIdx.x;
    const int tl = threadIdx.x;
    const int64_t ts = (int64_t)tt * TT + tl;
    const int4 tv = a.slot_v[ts];
    if (tv.x < 0) return;
    const int dom = tv.w;
    const int2 dr = a.dom_tiles[dom];
    int sb = blockIdx.y * a.chunk_tiles, se = min(sb + a.chunk_tiles, a.n_tiles);
    if (a.slot == 1) {
        sb = max(sb, dr.x);
        se = min(se, dr.y);
    }
    if (sb >= se) return;
    const double2 kd = a.slot == 0 ? a.k0 : a.kdom[dom];
    const double kr = kd.x, ki = kd.y;
    const SlotCoef cf = a.coef[dom * 2 + a.slot];
    const double inv4pi = 0.07957747154594767;
    const double4 ng = tg64[ts];
    const double4 ct = a.tc[tt];
    const int64_t ra[3] = {a.v_dof1[tv.x], a.v_dof1[tv.y], a.v_dof1[tv.z]};
    const int64_t rb[3] = {a.v_dof2[tv.x], a.v_dof2[tv.y], a.v_dof2[tv.z]};
    for (int s = sb; s < se; s++) {
        const double4 cs = a.tc[s];
        const double Dx = ct.x - cs.x, Dy = ct.y - cs.y, Dz = ct.z - cs.z;
        const int ntri = a.tntri[s];
        for (int sl = 0; sl < ntri; sl++) {
            const int64_t ss = (int64_t)s * TT + sl;
            if (ss == ts) continue;
            const double4 sg = tg64[ss];
            double V[3][3][2] = {}, K[3][3][2] = {}, Kp[3][3][2] = {};
            for (int qx = 0; qx < QP; qx++) {
                const double4 x = pg64[ts * QP + qx];
                const double Xx = x.x + Dx, Xy = x.y + Dy, Xz = x.z + Dz;  // x - c_source
                const double fK = sg.w - (sg.x * Xx + sg.y * Xy + sg.z * Xz);
                double hV[3][2] = {}, hK[3][2] = {}, hKp[3][2] = {};
                for (int qy = 0; qy < QP; qy++) {
                    const double4 y = pg64[ss * QP + qy];
                    const double ex = Xx - y.x, ey = Xy - y.y, ez = Xz - y.z;  // x - y
                    const double r = sqrt(ex * ex + ey * ey + ez * ez);
                    const double rinv = 1.0 / r;
                    double sn, c2;
                    sincos(kr * r, &sn, &c2);
                    const double am = exp(-ki * r) * rinv;
                    const double Gr = am * c2, Gi = am * sn;
                    const double u = -ki - rinv;
                    const double Fr = (Gr * u - Gi * kr) * rinv, Fi = (Gr * kr + Gi * u) * rinv;
                    const double ndot = ng.x * ex + ng.y * ey + ng.z * ez;
                    for (int b = 0; b < 3; b++) {
                        const double wl = y.w * (double)a.lam64[qy][b];
                        hV[b][0] += wl * Gr;
                        hV[b][1] += wl * Gi;
                        hK[b][0] += wl * Fr;
                        hK[b][1] += wl * Fi;
                        hKp[b][0] += wl * ndot * Fr;
                        hKp[b][1] += wl * ndot * Fi;
                    }
                }
                for (int i = 0; i < 3; i++) {
                    const double wx = x.w * a.lam64[qx][i] * inv4pi;
                    for (int b = 0; b < 3; b++) {
                        V[i][b][0] += wx * hV[b][0];
                        V[i][b][1] += wx * hV[b][1];
                        K[i][b][0] += wx * fK * hK[b][0];
                        K[i][b][1] += wx * fK * hK[b][1];
                        Kp[i][b][0] += wx * hKp[b][0];
                        Kp[i][b][1] += wx * hKp[b][1];
                    }
                }
            }
            double sr = 0, si = 0;
            for (int i = 0; i < 3; i++)
                for (int b = 0; b < 3; b++) {
                    sr += V[i][b][0];
                    si += V[i][b][1];
                }
            const double nn = ng.x * sg.x + ng.y * sg.y + ng.z * sg.z;
            const int4 sv = a.slot_v[ss];
            const int vb[3] = {sv.x, sv.y, sv.z};
            for (int b = 0; b < 3; b++) {
                const int64_t ca = a.v_dof1[vb[b]], cb = a.v_dof2[vb[b]];
                for (int i = 0; i < 3; i++) {
                    double cc = 0;
                    for (int c = 0; c < 3; c++) cc += a.slot_curl[ts * 9 + 3 * i + c] * a.slot_curl[ss * 9 + 3 * b + c];
                    const double kvr = cf.k2re * V[i][b][0] - cf.k2im * V[i][b][1];
                    const double kvi = cf.k2re * V[i][b][1] + cf.k2im * V[i][b][0];
                    double* e;
                    e = reinterpret_cast<double*>(&A64[ra[i] * a.n + ca]);
                    atomicAdd(e, cf.cV * V[i][b][0]);
                    atomicAdd(e + 1, cf.cV * V[i][b][1]);
                    e = reinterpret_cast<double*>(&A64[ra[i] * a.n + cb]);
                    atomicAdd(e, -cf.cK * K[i][b][0]);
                    atomicAdd(e + 1, -cf.cK * K[i][b][1]);
                    e = reinterpret_cast<double*>(&A64[rb[i] * a.n + ca]);
                    atomicAdd(e, cf.cKp * Kp[i][b][0]);
                    atomicAdd(e + 1, cf.cKp * Kp[i][b][1]);
                    e = reinterpret_cast<double*>(&A64[rb[i] * a.n + cb]);
                    atomicAdd(e, cf.cW * (cc * sr - nn * kvr));
                    atomicAdd(e + 1, cf.cW * (cc * si - nn * kvi));
                }
            }
        }
    }
}

// The same assembly with the kernel values and their P1 moments in
// double-float FP32 arithmetic (df_math.cuh), about 1e-13 relative, and the
// coefficient epilogue in FP64 from the converted moments: GB300 runs FP64 at
// ~1/64 of the FP32 rate, and the 36 point pairs of a triangle pair dominate.
struct AssembleDf {
    const float4 *pgh, *pgl, *tgh, *tgl, *tch, *tcl;  // split geometry (bem_ctx::ensure_fardf)
    const float4* kdf;        // [n_dom] (Re k hi, lo, Im k hi, lo)
    float4 k0df;
    const float4* sctab;
    const float2* extab;
    DfConsts c;
    float lamh[QP][3], laml[QP][3];  // P1 values at the rule points
    float i4h, i4l;                  // 1 / (4 pi)
};

template <bool ATTEN>
__device__ __forceinline__ void assembledf_body(const AssembleArgs& a, const AssembleDf& d, double2* A64,
                                                const float4* __restrict__ tab, const float2* __restrict__ etab) {
    const int tt = blockIdx.x;
    const int tl = threadIdx.x;
    const int64_t ts = (int64_t)tt * TT + tl;
    const int4 tv = a.slot_v[ts];
    if (tv.x < 0) return;
    const int dom = tv.w;
    const int2 dr = a.dom_tiles[dom];
    int sb = blockIdx.y * a.chunk_tiles, se = min(sb + a.chunk_tiles, a.n_tiles);
    if (a.slot == 1) {
        sb = max(sb, dr.x);
        se = min(se, dr.y);
    }
    if (sb >= se) return;
    const float4 kk = a.slot == 0 ? d.k0df : d.kdf[dom];
    const dfl kr = {kk.x, kk.y}, ki = {kk.z, kk.w};
    const SlotCoef cf = a.coef[dom * 2 + a.slot];
    const float4 nh = d.tgh[ts], nl = d.tgl[ts];
    const dfl ngx = {nh.x, nl.x}, ngy = {nh.y, nl.y}, ngz = {nh.z, nl.z};
    const float4 cth = d.tch[tt], ctl = d.tcl[tt];
    const int64_t ra[3] = {a.v_dof1[tv.x], a.v_dof1[tv.y], a.v_dof1[tv.z]};
    const int64_t rb[3] = {a.v_dof2[tv.x], a.v_dof2[tv.y], a.v_dof2[tv.z]};
    const dfl i4 = {d.i4h, d.i4l};
    for (int s = sb; s < se; s++) {
        const float4 csh = d.tch[s], csl = d.tcl[s];
        const dfl Dx = dsub(dfl{cth.x, ctl.x}, dfl{csh.x, csl.x});
        const dfl Dy = dsub(dfl{cth.y, ctl.y}, dfl{csh.y, csl.y});
        const dfl Dz = dsub(dfl{cth.z, ctl.z}, dfl{csh.z, csl.z});
        const int ntri = a.tntri[s];
        for (int sl = 0; sl < ntri; sl++) {
            const int64_t ss = (int64_t)s * TT + sl;
            if (ss == ts) continue;
            const float4 sgh = d.tgh[ss], sgl = d.tgl[ss];
            const dfl snx = {sgh.x, sgl.x}, sny = {sgh.y, sgl.y}, snz = {sgh.z, sgl.z}, sh = {sgh.w, sgl.w};
            dfl V[3][3][2], K[3][3][2], Kp[3][3][2];
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int b = 0; b < 3; b++)
#pragma unroll
                    for (int c = 0; c < 2; c++) V[i][b][c] = K[i][b][c] = Kp[i][b][c] = dfl{0.0f, 0.0f};
            for (int qx = 0; qx < QP; qx++) {
                const float4 xh = d.pgh[ts * QP + qx], xl = d.pgl[ts * QP + qx];
                const dfl Xx = dadd(dfl{xh.x, xl.x}, Dx), Xy = dadd(dfl{xh.y, xl.y}, Dy), Xz = dadd(dfl{xh.z, xl.z}, Dz);
                const dfl fK = dsub(sh, dadd(dadd(dmul(snx, Xx), dmul(sny, Xy)), dmul(snz, Xz)));
                dfl hV[3][2], hK[3][2], hKp[3][2];
#pragma unroll
                for (int b = 0; b < 3; b++)
#pragma unroll
                    for (int c = 0; c < 2; c++) hV[b][c] = hK[b][c] = hKp[b][c] = dfl{0.0f, 0.0f};
                for (int qy = 0; qy < QP; qy++) {
                    const float4 yh = d.pgh[ss * QP + qy], yl = d.pgl[ss * QP + qy];
                    const dfl ex = dsub(Xx, dfl{yh.x, yl.x}), ey = dsub(Xy, dfl{yh.y, yl.y}), ez = dsub(Xz, dfl{yh.z, yl.z});
                    dfl r, ri;
                    dsqrt_rinv(dadd(dadd(dsqr(ex), dsqr(ey)), dsqr(ez)), r, ri);
                    dfl sn, cs;
                    dsincos(dmul(kr, r), d.c, tab, sn, cs);
                    const dfl am = ATTEN ? dmul(dexp_neg(dmul(ki, r), d.c, etab), ri) : ri;
                    const dfl Gr = dmul(am, cs), Gi = dmul(am, sn);
                    const dfl u = dsub(dneg(ki), ri);
                    const dfl Fr = dmul(dsub(dmul(Gr, u), dmul(Gi, kr)), ri);
                    const dfl Fi = dmul(dadd(dmul(Gr, kr), dmul(Gi, u)), ri);
                    const dfl ndot = dadd(dadd(dmul(ngx, ex), dmul(ngy, ey)), dmul(ngz, ez));
                    const dfl nFr = dmul(ndot, Fr), nFi = dmul(ndot, Fi);
                    const dfl yw = {yh.w, yl.w};
#pragma unroll
                    for (int b = 0; b < 3; b++) {
                        const dfl wl = dmul(yw, dfl{d.lamh[qy][b], d.laml[qy][b]});
                        dmac(hV[b][0], wl, Gr, 1.0f);
                        dmac(hV[b][1], wl, Gi, 1.0f);
                        dmac(hK[b][0], wl, Fr, 1.0f);
                        dmac(hK[b][1], wl, Fi, 1.0f);
                        dmac(hKp[b][0], wl, nFr, 1.0f);
                        dmac(hKp[b][1], wl, nFi, 1.0f);
                    }
                }
                const dfl xw = dmul(dfl{xh.w, xl.w}, i4);
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const dfl wx = dmul(xw, dfl{d.lamh[qx][i], d.laml[qx][i]});
                    const dfl wk = dmul(wx, fK);
#pragma unroll
                    for (int b = 0; b < 3; b++)
#pragma unroll
                        for (int c = 0; c < 2; c++) {
                            dmac(V[i][b][c], wx, hV[b][c], 1.0f);
                            dmac(K[i][b][c], wk, hK[b][c], 1.0f);
                            dmac(Kp[i][b][c], wx, hKp[b][c], 1.0f);
                        }
                }
            }
            // epilogue in FP64 (as assemble64_kernel) from the converted moments
            double Vd[3][3][2];
            double sr = 0, si = 0;
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    Vd[i][b][0] = (double)V[i][b][0].h + (double)V[i][b][0].l;
                    Vd[i][b][1] = (double)V[i][b][1].h + (double)V[i][b][1].l;
                    sr += Vd[i][b][0];
                    si += Vd[i][b][1];
                }
            const double nn = ((double)ngx.h + ngx.l) * ((double)snx.h + snx.l) +
                              ((double)ngy.h + ngy.l) * ((double)sny.h + sny.l) +
                              ((double)ngz.h + ngz.l) * ((double)snz.h + snz.l);
            const int4 sv = a.slot_v[ss];
            const int vb[3] = {sv.x, sv.y, sv.z};
            for (int b = 0; b < 3; b++) {
                const int64_t ca = a.v_dof1[vb[b]], cb = a.v_dof2[vb[b]];
                for (int i = 0; i < 3; i++) {
                    double cc = 0;
                    for (int c = 0; c < 3; c++) cc += a.slot_curl[ts * 9 + 3 * i + c] * a.slot_curl[ss * 9 + 3 * b + c];
                    const double kvr = cf.k2re * Vd[i][b][0] - cf.k2im * Vd[i][b][1];
                    const double kvi = cf.k2re * Vd[i][b][1] + cf.k2im * Vd[i][b][0];
                    const double Kr = (double)K[i][b][0].h + (double)K[i][b][0].l;
                    const double Ki = (double)K[i][b][1].h + (double)K[i][b][1].l;
                    const double Pr = (double)Kp[i][b][0].h + (double)Kp[i][b][0].l;
                    const double Pi = (double)Kp[i][b][1].h + (double)Kp[i][b][1].l;
                    double* e;
                    e = reinterpret_cast<double*>(&A64[ra[i] * a.n + ca]);
                    atomicAdd(e, cf.cV * Vd[i][b][0]);
                    atomicAdd(e + 1, cf.cV * Vd[i][b][1]);
                    e = reinterpret_cast<double*>(&A64[ra[i] * a.n + cb]);
                    atomicAdd(e, -cf.cK * Kr);
                    atomicAdd(e + 1, -cf.cK * Ki);
                    e = reinterpret_cast<double*>(&A64[rb[i] * a.n + ca]);
                    atomicAdd(e, cf.cKp * Pr);
                    atomicAdd(e + 1, cf.cKp * Pi);
                    e = reinterpret_cast<double*>(&A64[rb[i] * a.n + cb]);
                    atomicAdd(e, cf.cW * (cc * sr - nn * kvr));
                    atomicAdd(e + 1, cf.cW * (cc * si - nn * kvi));
                }
            }
        }
    }
}

__global__ void __launch_bounds__(TT) assembledf_kernel(AssembleArgs a, AssembleDf d, double2* A64) {
    __shared__ float4 tab[128];
    __shared__ float2 etab[64];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) tab[i] = d.sctab[i];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) etab[i] = d.extab[i];
    __syncthreads();
    const int4 tv = a.slot_v[(int64_t)blockIdx.x * TT + threadIdx.x];
    const float4 kk = a.slot == 0 ? d.k0df : d.kdf[tv.x >= 0 ? tv.w : 0];
    if (kk.z != 0.0f || kk.w != 0.0f) assembledf_body<true>(a, d, A64, tab, etab);
    else assembledf_body<false>(a, d, A64, tab, etab);
}

__global__ void add_near64_kernel(int64_t n_pairs, const int32_t* pair_tgt, const int32_t* pair_src,
                                  const int4* slot_v, const int64_t* v_dof1, const int64_t* v_dof2,
                                  const double2* nb64, int64_t n, double2* A) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const int4 tv = slot_v[pair_tgt[p]], sv = slot_v[pair_src[p]];
    const int va[3] = {tv.x, tv.y, tv.z}, vb[3] = {sv.x, sv.y, sv.z};
    for (int blk = 0; blk < 4; blk++)
        for (int i = 0; i < 3; i++)
            for (int b = 0; b < 3; b++) {
                const int64_t row = (blk < 2) ? v_dof1[va[i]] : v_dof2[va[i]];
                const int64_t col = (blk & 1) ? v_dof2[vb[b]] : v_dof1[vb[b]];
                const double2 v = nb64[(p * 4 + blk) * 9 + 3 * i + b];
                double* e = reinterpret_cast<double*>(&A[row * n + col]);
                atomicAdd(e, v.x);
                atomicAdd(e + 1, v.y);
            }
}

// Touching-pair corrections (combined FP32 blocks) into the dense matrix.
__global__ void add_near_kernel(int64_t n_pairs, const int32_t* pair_tgt, const int32_t* pair_src, const int4* slot_v,
                                const int64_t* v_dof1, const int64_t* v_dof2, const float2* nb32, int64_t n,
                                float2* A) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pairs) return;
    const int4 tv = slot_v[pair_tgt[p]], sv = slot_v[pair_src[p]];
    const int va[3] = {tv.x, tv.y, tv.z}, vb[3] = {sv.x, sv.y, sv.z};
    for (int blk = 0; blk < 4; blk++)
        for (int i = 0; i < 3; i++)
            for (int b = 0; b < 3; b++) {
                const int64_t row = (blk < 2) ? v_dof1[va[i]] : v_dof2[va[i]];
                const int64_t col = (blk & 1) ? v_dof2[vb[b]] : v_dof1[vb[b]];
                atomicAdd(&A[row * n + col], nb32[(p * 4 + blk) * 9 + 3 * i + b]);
            }
}

__global__ void c128_to_c64(int64_t n, const double2* x, float2* y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = make_float2((float)x[i].x, (float)x[i].y);
}

__global__ void c64_to_c128(int64_t n, const float2* x, double2* y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = make_double2(x[i].x, x[i].y);
}

int gemm_bf16x3(bem_ctx* ctx, const __nv_bfloat16* Aplanes, int64_t m, int64_t k, int64_t mpad, int64_t kpad,
                const float2* X, int64_t n_rhs, float2* Y, __nv_bfloat16* xplanes, int64_t nbpad);
int split_a(bem_ctx* ctx, const float2* A, int64_t m, int64_t k, int64_t mpad, int64_t kpad, __nv_bfloat16* P);
int gemm_a_planes();
int gemm_b_planes();
int gemm_k_align();

}  // namespace gbem

using namespace gbem;

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// Assemble A_hat (complex64, dense) and its split-BF16 planes; cached in ctx.
int bem_ctx::ensure_assembled() {
    bem_ctx* const ctx = this;
    if (asm_ready) return BEM_OK;
    int rc = ensure_near();
    if (rc) return rc;
    const Geometry& g = geo;
    const int64_t n = g.n_dof;
    const int64_t ka = gemm_k_align();
    const int64_t mpad = (n + 127) / 128 * 128, kpad = (n + ka - 1) / ka * ka;
    if (asm_planes) { dfree(asm_planes); asm_planes = nullptr; }
    float2* A = (float2*)dalloc((size_t)n * n * sizeof(float2), &rc);
    if (rc) return rc;
    CK(cudaMemsetAsync(A, 0, (size_t)n * n * sizeof(float2), stream));
    AssembleArgs a{};
    a.pg = dev.pg32; a.tg = dev.tg32; a.tc = dev.tc; a.tntri = dev.tntri; a.slot_v = dev.slot_v;
    a.slot_curl = dev.slot_curl; a.v_dof1 = dev.v_dof1; a.v_dof2 = dev.v_dof2; a.coef = dev.coef;
    a.dom_tiles = dev.dom_tiles; a.kdom = dev.kdom; a.k0 = make_double2(k0re, k0im);
    a.n_tiles = g.n_tiles; a.chunk_tiles = 16; a.n = n; a.A = A;
    for (int q = 0; q < QP; q++)
        for (int k = 0; k < 3; k++) {
            a.lam[q][k] = (float)quad.lam[q][k];
            a.lam64[q][k] = quad.lam[q][k];
        }
    const dim3 grid(g.n_tiles, (g.n_tiles + a.chunk_tiles - 1) / a.chunk_tiles);
    for (int sl = 0; sl < 2; sl++) {
        a.slot = sl;
        assemble_kernel<<<grid, TT, 0, stream>>>(a);
        CK(cudaGetLastError());
    }
    const int64_t np = pmchwt_near.n_pairs;
    if (np > 0) {
        add_near_kernel<<<(unsigned)((np + 127) / 128), 128, 0, stream>>>(np, dev.np_tgt, dev.np_src, dev.slot_v, dev.v_dof1,
                                                                         dev.v_dof2, pmchwt_near.nb32, n, A);
        CK(cudaGetLastError());
    }
    asm_planes = (__nv_bfloat16*)dalloc((size_t)gemm_a_planes() * mpad * kpad * 2, &rc);
    if (rc) { dfree(A); return rc; }
    if ((rc = split_a(this, A, n, n, mpad, kpad, asm_planes))) { dfree(A); return rc; }
    CK(cudaStreamSynchronize(stream));
    dfree(A);
    launches += 4;
    asm_mpad = mpad;
    asm_kpad = kpad;
    asm_ready = true;
    return BEM_OK;
}

// A_hat assembled in complex128 (FP64 arithmetic), kept for the FP64
// residual of the refinement: one pass of FP64 interactions at set-up, then
// the matrix is stored as scaled FP32 (hi, lo) pairs in the same 16 bytes per
// entry, and every residual is a product to FP64 accuracy in FP32 arithmetic
// that streams it at the HBM rate (k_df64.cu).
int bem_ctx::ensure_assembled64() {
    bem_ctx* const ctx = this;
    if (asm64_ready) return BEM_OK;
    int rc = ensure_near();
    if (rc) return rc;
    const Geometry& g = geo;
    const int64_t n = g.n_dof;
    if (asm64) { dfree(asm64); asm64 = nullptr; }
    asm64 = (double2*)dalloc((size_t)n * n * sizeof(double2), &rc);
    if (rc) { asm64 = nullptr; return rc; }
    CK(cudaMemsetAsync(asm64, 0, (size_t)n * n * sizeof(double2), stream));
    AssembleArgs a{};
    a.tc = dev.tc; a.tntri = dev.tntri; a.slot_v = dev.slot_v; a.slot_curl = dev.slot_curl;
    a.v_dof1 = dev.v_dof1; a.v_dof2 = dev.v_dof2; a.coef = dev.coef; a.dom_tiles = dev.dom_tiles; a.kdom = dev.kdom;
    a.k0 = make_double2(k0re, k0im); a.n_tiles = g.n_tiles; a.chunk_tiles = 8; a.n = n;
    for (int q = 0; q < QP; q++)
        for (int k = 0; k < 3; k++) a.lam64[q][k] = quad.lam[q][k];
    const dim3 grid(g.n_tiles, (g.n_tiles + a.chunk_tiles - 1) / a.chunk_tiles);
    AssembleDf d{};
    if (opts.fp64_far == 0) {  // double-float kernel values (the default), else native FP64
        if ((rc = ensure_fardf()) || (rc = check_df_phase(k0re, false))) return rc;
        d.pgh = dfg.pgh; d.pgl = dfg.pgl; d.tgh = dfg.tgh; d.tgl = dfg.tgl; d.tch = dfg.tch; d.tcl = dfg.tcl;
        d.kdf = dfg.kdf; d.sctab = dfg.sctab; d.extab = dfg.extab; d.c = dfg.c;
        auto split = [](long double v, float& h, float& l) {
            h = (float)v;
            l = (float)(v - (long double)h);
        };
        float h, l, ih, il;
        split((long double)k0re, h, l);
        split((long double)k0im, ih, il);
        d.k0df = make_float4(h, l, ih, il);
        for (int q = 0; q < QP; q++)
            for (int k = 0; k < 3; k++) split((long double)quad.lam[q][k], d.lamh[q][k], d.laml[q][k]);
        split(1.0L / (4.0L * 3.141592653589793238462643383279502884L), d.i4h, d.i4l);
    }
    for (int sl = 0; sl < 2; sl++) {
        a.slot = sl;
        if (opts.fp64_far == 0) assembledf_kernel<<<grid, TT, 0, stream>>>(a, d, asm64);
        else assemble64_kernel<<<grid, TT, 0, stream>>>(a, dev.pg64, dev.tg64, asm64);
        CK(cudaGetLastError());
    }
    const int64_t np = pmchwt_near.n_pairs;
    if (np > 0) {
        add_near64_kernel<<<(unsigned)((np + 127) / 128), 128, 0, stream>>>(np, dev.np_tgt, dev.np_src, dev.slot_v,
                                                                           dev.v_dof1, dev.v_dof2, pmchwt_near.nb64,
                                                                           n, asm64);
        CK(cudaGetLastError());
    }
    CK(cudaGetLastError());
    if (!df_exp) {
        df_exp = (int*)dalloc(2 * sizeof(int), &rc);
        if (rc) { df_exp = nullptr; return rc; }
    }
    if ((rc = df_prepare_inplace(this, asm64, n * n, df_exp))) return rc;
    CK(cudaStreamSynchronize(stream));
    launches += 3;
    asm64_ready = true;
    return BEM_OK;
}

// Y = A_hat X (FP64 accuracy, assembled) for n_rhs system-order vectors;
// A_hat is row-major in the split form of k_df64.cu.
int bem_ctx::apply_assembled64(const double2* x, double2* y, int64_t n_rhs) {
    int rc = ensure_assembled64();
    if (rc) return rc;
    const int64_t n = geo.n_dof;
    return df_gemv(this, (const float4*)asm64, df_exp, n, n, n, x, n_rhs, y, n);
}

// Y = A_hat X for n_rhs system-order vectors (complex128, device), through
// the assembled operator and the tensor-core GEMM.
int bem_ctx::apply_assembled(const double2* x, double2* y, int64_t n_rhs) {
    bem_ctx* const ctx = this;
    int rc = ensure_assembled();
    if (rc) return rc;
    const int64_t n = geo.n_dof;
    const int64_t nbpad = (n_rhs + 63) / 64 * 128;
    const size_t need = (size_t)n_rhs * n * sizeof(float2) * 2 + (size_t)gemm_b_planes() * nbpad * asm_kpad * 2;
    if (need > asm_work_bytes) {
        if (asm_work) dfree(asm_work);
        asm_work = dalloc(need, &rc);
        if (rc) { asm_work = nullptr; asm_work_bytes = 0; return rc; }
        asm_work_bytes = need;
    }
    float2* xs = (float2*)asm_work;
    float2* ys = xs + n_rhs * n;
    __nv_bfloat16* xp = (__nv_bfloat16*)(ys + n_rhs * n);
    const int64_t tot = n_rhs * n;
    c128_to_c64<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(tot, x, xs);
    if ((rc = gemm_bf16x3(this, asm_planes, n, n, asm_mpad, asm_kpad, xs, n_rhs, ys, xp, nbpad))) return rc;
    c64_to_c128<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(tot, ys, y);
    launches += 2;
    CK(cudaGetLastError());
    return BEM_OK;
}
