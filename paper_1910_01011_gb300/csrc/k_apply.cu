// k_apply.cu -- matrix-free application of the Galerkin boundary operators.
//
// Paper App. A (eqs. SLP, DLP, ADJDLP, HYP, green_func) and Sec. 2.3 (eq.
// Galerkin_disc_lhs): with G = exp(ikr)/(4 pi r), F = G (ik - 1/r)/r and P1
// trial data phi (Dirichlet) and psi (Neumann), the potentials at a target
// quadrature point x are
//   P_V   = sum_y G       w_y psi(y)                       (single layer)
//   P_K   = sum_y F (y-x).n_y w_y phi(y)                   (double layer)
//   P_K'  = sum_y F (x-y).n_x w_y psi(y)                   (adjoint double layer)
//   P_Wc  = sum_y G w_y curl phi(y),  P_Wm = sum_y G (n_x.n_y) w_y phi(y)
// (the hypersingular operator in its integration-by-parts form), and the
// Galerkin rows follow by testing with the P1 functions at the target
// points.  Per trial triangle t the plane offset (y-x).n_t and n_x.n_t are
// constant, and curl phi is constant, so three per-triangle sums
// S1 = sum F sigma_D, S2 = sum G w, S3 = sum G sigma_D carry K and W.
//
// The FP32 kernel keeps kr accurate for large k|x-y| by reconstructing the
// distance from the tile-pair centre distance R_c (FP64) and a local
// offset: with D = c_target - c_source and delta = dx - dy (tile-local),
//   s = delta.(2D + delta) = r^2 - R_c^2,   r - R_c = s / (r + R_c),
//   phase = (Re k R_c mod 2 pi, FP64) + Re k (r - R_c).
#include <cstdio>

#include "internal.h"
#include "pair_math.h"

namespace gbem {

// ----------------------------------------------------------------- helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok;
}

// Bulk (TMA) copy global -> shared completing on an mbarrier.  Both
// addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait: gives up after ~2^31 cycles (about a second), raises the
// device error flag and lets the caller continue on whatever the buffer
// holds, so that every thread still reaches every __syncthreads.
__device__ __forceinline__ void mbar_wait_bounded(uint64_t* b, uint32_t parity, int* err) {
    if (mbar_try_wait(b, parity)) return;
    long long t0 = clock64();
    while (!mbar_try_wait(b, parity)) {
        if (clock64() - t0 > (1ll << 31)) {
            atomicExch(err, 1);
            return;
        }
    }
}

// x - 2 pi round(x / 2 pi) in FP64 (2 pi split in two doubles), as float.
__device__ __forceinline__ float reduce_phase(double t) {
    const double two_pi_hi = 6.283185307179586, two_pi_lo = 2.4492935982947064e-16;
    double n = rint(t * 0.15915494309189535);
    double r = fma(-n, two_pi_hi, t);
    r = fma(-n, two_pi_lo, r);
    return (float)r;
}


// ----------------------------------------------------------------- gather (trial densities)

__global__ void gather_kernel(GatherArgs a) {
    const int64_t s = a.s_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.s_end) return;
    int4 v = a.slot_v[s];
    double2 xs[3], xf[3];
    bool real = v.x >= 0;
    for (int k = 0; k < 3; k++) {
        int vid = k == 0 ? v.x : k == 1 ? v.y : v.z;
        if (real) {
            xs[k] = a.x[a.v_dof1[vid]];
            xf[k] = a.x[a.v_dof2[vid]];
        } else {
            xs[k] = make_double2(0, 0);
            xf[k] = make_double2(0, 0);
        }
    }
    float4 p32[QP];
    for (int q = 0; q < QP; q++) {
        double w = real ? a.pt_w[s * QP + q] : 0.0;
        double sr = 0, si = 0, dr = 0, di = 0;
        for (int k = 0; k < 3; k++) {
            sr += a.lam[q][k] * xs[k].x;
            si += a.lam[q][k] * xs[k].y;
            dr += a.lam[q][k] * xf[k].x;
            di += a.lam[q][k] * xf[k].y;
        }
        p32[q] = make_float4((float)(w * sr), (float)(w * si), (float)(w * dr), (float)(w * di));
        if (a.pd64) a.pd64[s * QP + q] = make_double4(w * sr, w * si, w * dr, w * di);
    }
    if (a.pd32) pair_interleave(p32, a.pd32 + s * QP);
    double cr[3] = {0, 0, 0}, ci[3] = {0, 0, 0};
    if (real)
        for (int k = 0; k < 3; k++)
            for (int c = 0; c < 3; c++) {
                double cu = a.slot_curl[s * 9 + 3 * k + c];
                cr[c] += xf[k].x * cu;
                ci[c] += xf[k].y * cu;
            }
    if (a.tcurl32) {
        a.tcurl32[2 * s] = make_float4((float)cr[0], (float)cr[1], (float)cr[2], 0.f);
        a.tcurl32[2 * s + 1] = make_float4((float)ci[0], (float)ci[1], (float)ci[2], 0.f);
    }
    if (a.tcurl64) {
        a.tcurl64[2 * s] = make_double4(cr[0], cr[1], cr[2], 0.0);
        a.tcurl64[2 * s + 1] = make_double4(ci[0], ci[1], ci[2], 0.0);
    }
}

// ----------------------------------------------------------------- FP32 far field
//
// One CTA = one target tile (TP threads, one target point each) against a
// contiguous range of source tiles.  Source tiles stream through an
// NSTAGE-deep ring of shared-memory stages filled by bulk (TMA) copies that
// complete on per-stage mbarriers.  There is no CTA-wide barrier in the
// loop: each warp counts itself out of a stage when it has finished the
// tile in it, and the last warp to leave a stage refills it with the tile
// NSTAGE ahead, so warps drift freely within the ring.

constexpr int NSTAGE = 4;
constexpr int NWARP = TP / 32;

struct __align__(16) Stage {
    float4 pg[TP];      // source points (dx, dy, dz, w), pair-interleaved
    float4 pd[TP];      // densities, pair-interleaved
    float4 tg[TT];      // triangles (n, h)
    float4 tc[2 * TT];  // curl densities
};
constexpr uint32_t STAGE_BYTES = sizeof(Stage);
static_assert(STAGE_BYTES == 7680, "stage layout");

struct FarSmem {
    Stage st[NSTAGE];
    float4 tab[2 * CHUNK_MAX];
    uint64_t full[NSTAGE];
    int cnt[NSTAGE];
};

struct Acc {
    float v[NCOMP];  // PV(2) PK(2) PKp(2) PWm(2) PWc(6)
};

// Source points are processed two at a time, side by side in the two lanes
// of a float2, so that one packed FP32 instruction (FFMA2 / FADD2 / FMUL2)
// advances both.  The points of a triangle are stored pair-interleaved:
// pair j (points 2j and 2j+1) is the float4 (x_a, x_b, y_a, y_b) followed by
// (z_a, z_b, w_a, w_b), for the source geometry (offsets from the tile
// centre and weight) and for the gathered densities (the two complex
// densities in place of x, y and z, w).  The packed helpers are in
// pair_math.h.

// One wavenumber slot, both lanes.
struct PairK {
    f2 kr, nkr, th, ki, nkil2;  // Re k, -Re k, reduced FP64 phase of the tile pair, Im k, -Im k log2(e)
};

// Sums over the points of one tile (V, K') and of one triangle (the rest),
// per lane; they are folded into the chunk's accumulators at the end of
// their tile or triangle.  The K' and K sums are kept with the sign of -F,
// the form in which the gradient factor comes out without a sign flip.
struct PairTile {
    f2 Vr, Vi, nKpr, nKpi;
};
struct PairTri {
    f2 nS1r, nS1i, S2r, S2i, S3r, S3i;
};

// Contribution of two source points at one wavenumber.  With
// (ik - 1/r)/r = A + iB, B = Re k / r, P = -A = Im k / r + 1/r^2, the
// gradient factor is F = G (A + iB), so -Re F = P Gr + B Gi and
// -Im F = P Gi - B Gr.  LOSSY: Im k != 0 (exp(-Im k r) evaluated);
// otherwise the amplitude is 1/r and P = 1/r^2.
template <bool LOSSY>
__device__ __forceinline__ void pair_slot(const PairK& k, f2 rho, f2 r, f2 rinv, f2 rinv2, f2 ndot, f2 w, f2 d1r,
                                          f2 d1i, f2 nd1i, f2 d2r, f2 d2i, f2 nd2i, PairTile& T, PairTri& S) {
    const f2 arg = fma2(k.kr, rho, k.th);
    f2 sn, cs;
    sincos_approx(arg.x, &sn.x, &cs.x);
    sincos_approx(arg.y, &sn.y, &cs.y);
    f2 a = rinv;
    if constexpr (LOSSY) {
        const f2 e = mul2(k.nkil2, r);
        a = mul2(make_float2(ex2_approx(e.x), ex2_approx(e.y)), rinv);
    }
    const f2 Gr = mul2(a, cs), Gi = mul2(a, sn);
    const f2 B = mul2(k.kr, rinv), nB = mul2(k.nkr, rinv);
    const f2 P = LOSSY ? fma2(k.ki, rinv, rinv2) : rinv2;
    const f2 nFr = fma2(P, Gr, mul2(B, Gi));
    const f2 nFi = fma2(P, Gi, mul2(nB, Gr));
    T.Vr = fma2(Gr, d1r, fma2(Gi, nd1i, T.Vr));
    T.Vi = fma2(Gr, d1i, fma2(Gi, d1r, T.Vi));
    const f2 nFnr = mul2(ndot, nFr), nFni = mul2(ndot, nFi);
    T.nKpr = fma2(nFnr, d1r, fma2(nFni, nd1i, T.nKpr));
    T.nKpi = fma2(nFnr, d1i, fma2(nFni, d1r, T.nKpi));
    S.nS1r = fma2(nFr, d2r, fma2(nFi, nd2i, S.nS1r));
    S.nS1i = fma2(nFr, d2i, fma2(nFi, d2r, S.nS1i));
    S.S2r = fma2(Gr, w, S.S2r);
    S.S2i = fma2(Gi, w, S.S2i);
    S.S3r = fma2(Gr, d2r, fma2(Gi, nd2i, S.S3r));
    S.S3i = fma2(Gr, d2i, fma2(Gi, d2r, S.S3i));
}

// Per-triangle terms: K through (y-x).n_t, W through curl phi and n_x.n_t.
__device__ __forceinline__ void slot_triangle(float fK, float nn, const float4& cre, const float4& cim,
                                              const PairTri& P, Acc& t) {
    const float nS1r = P.nS1r.x + P.nS1r.y, nS1i = P.nS1i.x + P.nS1i.y;
    const float S2r = P.S2r.x + P.S2r.y, S2i = P.S2i.x + P.S2i.y;
    const float S3r = P.S3r.x + P.S3r.y, S3i = P.S3i.x + P.S3i.y;
    t.v[2] = fmaf(-fK, nS1r, t.v[2]);
    t.v[3] = fmaf(-fK, nS1i, t.v[3]);
    t.v[6] = fmaf(nn, S3r, t.v[6]);
    t.v[7] = fmaf(nn, S3i, t.v[7]);
    t.v[8] = fmaf(S2r, cre.x, fmaf(-S2i, cim.x, t.v[8]));
    t.v[9] = fmaf(S2r, cre.y, fmaf(-S2i, cim.y, t.v[9]));
    t.v[10] = fmaf(S2r, cre.z, fmaf(-S2i, cim.z, t.v[10]));
    t.v[11] = fmaf(S2r, cim.x, fmaf(S2i, cre.x, t.v[11]));
    t.v[12] = fmaf(S2r, cim.y, fmaf(S2i, cre.y, t.v[12]));
    t.v[13] = fmaf(S2r, cim.z, fmaf(S2i, cre.z, t.v[13]));
}

// The target point of a thread: offset d from its tile centre, normal n,
// with -n and |d|^2, n.d kept for the per-tile constants.
struct PairTgt {
    float dx, dy, dz, nx, ny, nz, dd, nd;
    f2 nnx, nny, nnz;
};

// One target point against one source tile.  With D = c_target - c_source
// (c0 carries 2D and R_c^2 = |D|^2, c1 R_c and the reduced phases), a source
// point offset g from its centre gives x - y = d - g + D and
//   s = r^2 - R_c^2 = |g|^2 - 2 g.(d + D) + |d|^2 + 2 D.d,
// a sum whose terms are as small as s itself times R_c / tile size, so that
// the phase offset r - R_c = s / (r + R_c) keeps FP32 accuracy;
// n_x.(x - y) = (n.d + n.D) - n.g.
template <bool TWO, bool L0, bool L1>
__device__ __forceinline__ void tile_body(const Stage& st, int ntri, int skip_tl, const PairTgt& X, float4 c0, float4 c1,
                                          PairK k0, PairK k1, Acc& a0, Acc& a1) {
    const float D2x = c0.x, D2y = c0.y, D2z = c0.z;
    const f2 m2x = bc2(-fmaf(2.f, X.dx, D2x)), m2y = bc2(-fmaf(2.f, X.dy, D2y)), m2z = bc2(-fmaf(2.f, X.dz, D2z));
    const f2 cb = bc2(fmaf(D2x, X.dx, fmaf(D2y, X.dy, fmaf(D2z, X.dz, X.dd))));
    const f2 cn = bc2(fmaf(0.5f, X.nx * D2x + X.ny * D2y + X.nz * D2z, X.nd));
    const f2 Rc2 = bc2(c0.w), Rc = bc2(c1.x);
    k0.th = bc2(c1.y);
    if constexpr (TWO) k1.th = bc2(c1.z);
    const float Xx = fmaf(0.5f, D2x, X.dx), Xy = fmaf(0.5f, D2y, X.dy), Xz = fmaf(0.5f, D2z, X.dz);  // x - c_source
    const f2 z2 = make_float2(0.f, 0.f);
    PairTile T0{z2, z2, z2, z2}, T1{z2, z2, z2, z2};
    for (int tl = 0; tl < ntri; tl++) {
        if (tl == skip_tl) continue;  // identical triangle: near-field correction only
        PairTri S0{z2, z2, z2, z2, z2, z2}, S1{z2, z2, z2, z2, z2, z2};
#pragma unroll
        for (int j = 0; j < QP / 2; j++) {
            const float4 GA = st.pg[tl * QP + 2 * j], GB = st.pg[tl * QP + 2 * j + 1];
            const float4 DA = st.pd[tl * QP + 2 * j], DB = st.pd[tl * QP + 2 * j + 1];
            const f2 gx = lo2(GA), gy = hi2(GA), gz = lo2(GB), w = hi2(GB);
            const f2 d1r = lo2(DA), d1i = hi2(DA), d2r = lo2(DB), d2i = hi2(DB);
            const f2 s = fma2(gx, add2(gx, m2x), fma2(gy, add2(gy, m2y), fma2(gz, add2(gz, m2z), cb)));
            const f2 r2 = add2(s, Rc2);
            const f2 rinv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
            const f2 rinv2 = mul2(rinv, rinv);
            const f2 den = fma2(r2, rinv, Rc);  // r + R_c
            const f2 rho = mul2(s, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
            const f2 ndot = fma2(X.nnx, gx, fma2(X.nny, gy, fma2(X.nnz, gz, cn)));
            const f2 r = (L0 || L1) ? mul2(r2, rinv) : z2;
            const f2 nd1i = neg2(d1i), nd2i = neg2(d2i);
            pair_slot<L0>(k0, rho, r, rinv, rinv2, ndot, w, d1r, d1i, nd1i, d2r, d2i, nd2i, T0, S0);
            if constexpr (TWO) pair_slot<L1>(k1, rho, r, rinv, rinv2, ndot, w, d1r, d1i, nd1i, d2r, d2i, nd2i, T1, S1);
        }
        const float4 tg = st.tg[tl];
        const float4 cre = st.tc[2 * tl], cim = st.tc[2 * tl + 1];
        const float fK = tg.w - (tg.x * Xx + tg.y * Xy + tg.z * Xz);  // n_t.(y - x)
        const float nn = X.nx * tg.x + X.ny * tg.y + X.nz * tg.z;      // n_x.n_t
        slot_triangle(fK, nn, cre, cim, S0, a0);
        if constexpr (TWO) slot_triangle(fK, nn, cre, cim, S1, a1);
    }
    a0.v[0] += T0.Vr.x + T0.Vr.y;
    a0.v[1] += T0.Vi.x + T0.Vi.y;
    a0.v[4] -= T0.nKpr.x + T0.nKpr.y;
    a0.v[5] -= T0.nKpi.x + T0.nKpi.y;
    if constexpr (TWO) {
        a1.v[0] += T1.Vr.x + T1.Vr.y;
        a1.v[1] += T1.Vi.x + T1.Vi.y;
        a1.v[4] -= T1.nKpr.x + T1.nKpr.y;
        a1.v[5] -= T1.nKpi.x + T1.nKpi.y;
    }
}

// One work item: target tile tx (offset from A.tgt_begin) against source chunk cy.
__device__ __forceinline__ void far32_item(const FarArgs32& A, int tx, int cy) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FarSmem& sm = *reinterpret_cast<FarSmem*>(smem_raw);

    const int tid = threadIdx.x, lane = tid & 31;
    const int tt = A.tgt_begin + tx;
    const int sb = A.src_begin + cy * A.chunk_tiles;
    const int se = min(sb + A.chunk_tiles, A.src_end);
    const int nsrc = max(0, se - sb);

    const int64_t p = (int64_t)tt * TP + tid;
    const float4 g = A.pg[p];
    const int mt = tid / QP;
    const float4 ng = A.tg[(int64_t)tt * TT + mt];
    const double4 ct = A.tc[tt];
    const int mydom = A.tdom[tt];
    const int2 dr = A.dom_tiles[mydom];
    const double2 kj = A.kdom[mydom];
    const PairK k0{bc2((float)A.k0.x), bc2((float)-A.k0.x), bc2(0.f), bc2((float)A.k0.y),
                   bc2((float)(-A.k0.y * 1.4426950408889634))};
    const PairK k1{bc2((float)kj.x), bc2((float)-kj.x), bc2(0.f), bc2((float)kj.y),
                   bc2((float)(-kj.y * 1.4426950408889634))};
    const bool lossy0 = A.k0.y != 0.0, lossy1 = kj.y != 0.0;
    const PairTgt X{g.x, g.y, g.z, ng.x, ng.y, ng.z, g.x * g.x + g.y * g.y + g.z * g.z,
                    ng.x * g.x + ng.y * g.y + ng.z * g.z, bc2(-ng.x), bc2(-ng.y), bc2(-ng.z)};

    // tile-pair table: 2D, R_c^2, R_c and the FP64-reduced phases
    for (int i = tid; i < nsrc; i += TP) {
        const int s = sb + i;
        const double4 cs = A.tc[s];
        const double Dx = ct.x - cs.x, Dy = ct.y - cs.y, Dz = ct.z - cs.z;
        const double R = sqrt(Dx * Dx + Dy * Dy + Dz * Dz);
        const bool own = A.slot1 && s >= dr.x && s < dr.y;
        sm.tab[2 * i] = make_float4((float)(2 * Dx), (float)(2 * Dy), (float)(2 * Dz), (float)(R * R));
        sm.tab[2 * i + 1] = make_float4((float)R, reduce_phase(A.k0.x * R), own ? reduce_phase(kj.x * R) : 0.f, 0.f);
    }
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; s++) {
            mbar_init(&sm.full[s], 1);
            sm.cnt[s] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int i, int st) {
        const int s = sb + i;
        Stage& S = sm.st[st];
        mbar_arrive_expect_tx(&sm.full[st], STAGE_BYTES);
        bulk_g2s(S.pg, A.pgp + (int64_t)s * TP, TP * 16, &sm.full[st]);
        bulk_g2s(S.pd, A.pd + (int64_t)s * TP, TP * 16, &sm.full[st]);
        bulk_g2s(S.tg, A.tg + (int64_t)s * TT, TT * 16, &sm.full[st]);
        bulk_g2s(S.tc, A.tcurl + (int64_t)s * 2 * TT, 2 * TT * 16, &sm.full[st]);
    };
    if (tid == 0)
        for (int i = 0; i < min(NSTAGE, nsrc); i++) issue(i, i);

    Acc a0, a1;
#pragma unroll
    for (int c = 0; c < NCOMP; c++) {
        a0.v[c] = 0.f;
        a1.v[c] = 0.f;
    }
    for (int i = 0; i < nsrc; i++) {
        const int st = i % NSTAGE;
        mbar_wait_bounded(&sm.full[st], (uint32_t)((i / NSTAGE) & 1), A.err);
        const int s = sb + i;
        const Stage& S = sm.st[st];
        const int ntri = A.tntri[s];
        const int skip = (s == tt) ? mt : -1;
        const float4 c0 = sm.tab[2 * i], c1 = sm.tab[2 * i + 1];
        const bool two = A.slot1 && s >= dr.x && s < dr.y;
        if (two) {
            if (lossy0) {
                if (lossy1) tile_body<true, true, true>(S, ntri, skip, X, c0, c1, k0, k1, a0, a1);
                else tile_body<true, true, false>(S, ntri, skip, X, c0, c1, k0, k1, a0, a1);
            } else {
                if (lossy1) tile_body<true, false, true>(S, ntri, skip, X, c0, c1, k0, k1, a0, a1);
                else tile_body<true, false, false>(S, ntri, skip, X, c0, c1, k0, k1, a0, a1);
            }
        } else {
            if (lossy0) tile_body<false, true, false>(S, ntri, skip, X, c0, c1, k0, k1, a0, a1);
            else tile_body<false, false, false>(S, ntri, skip, X, c0, c1, k0, k1, a0, a1);
        }
        // leave the stage; the last warp out refills it with the tile NSTAGE ahead
        __syncwarp();
        if (lane == 0) {
            const int old = atomicAdd(&sm.cnt[st], 1);
            if (old == NWARP - 1) {
                sm.cnt[st] = 0;
                if (i + NSTAGE < nsrc) issue(i + NSTAGE, st);
            }
        }
    }

    float* out = A.partial + (int64_t)cy * 2 * NCOMP * A.n_pts + (p - A.p_off);
#pragma unroll
    for (int c = 0; c < NCOMP; c++) {
        out[(int64_t)c * A.n_pts] = a0.v[c];
        out[(int64_t)(NCOMP + c) * A.n_pts] = a1.v[c];
    }
}

__global__ void __launch_bounds__(TP, 2) far32_kernel(FarArgs32 A) {
    int tx = blockIdx.x, cy = blockIdx.y;
    if (A.work) {
        const int2 w = A.work[blockIdx.x];
        tx = w.x;
        cy = w.y;
    }
    far32_item(A, tx, cy);
}

// Several meshes in one launch: work item blockIdx.x is (mesh, target tile,
// chunk) = gwork[blockIdx.x], and the mesh's arguments are group[mesh].
__global__ void __launch_bounds__(TP, 2) far32_group_kernel(const FarArgs32* __restrict__ group,
                                                            const int4* __restrict__ gwork) {
    const int4 w = gwork[blockIdx.x];
    const FarArgs32 A = group[w.x];
    far32_item(A, w.y, w.z);
}

size_t far32_smem_bytes() { return sizeof(FarSmem); }

cudaError_t launch_far32(const FarArgs32& a, int n_tgt_tiles, int n_chunks, cudaStream_t s) {
    const size_t smem = far32_smem_bytes();
    static const cudaError_t attr_e =
        cudaFuncSetAttribute(far32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr_e != cudaSuccess) return attr_e;
    if (n_tgt_tiles <= 0 || n_chunks <= 0) return cudaSuccess;
    if (a.work) far32_kernel<<<(unsigned)((int64_t)n_tgt_tiles * n_chunks), TP, smem, s>>>(a);
    else far32_kernel<<<dim3(n_tgt_tiles, n_chunks), TP, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_far32_group(const FarArgs32* group, const int4* gwork, int64_t n_work, cudaStream_t s) {
    const size_t smem = far32_smem_bytes();
    static const cudaError_t attr_e =
        cudaFuncSetAttribute(far32_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr_e != cudaSuccess) return attr_e;
    if (n_work <= 0) return cudaSuccess;
    far32_group_kernel<<<(unsigned)n_work, TP, smem, s>>>(group, gwork);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- FP32 far field, several right-hand sides
//
// The Green's function G and the gradient factor F of a (target point,
// source point) pair do not depend on the densities, so a work item that
// serves MRG right-hand sides evaluates the geometry, the phase and the MUFU
// functions once and accumulates MRG sets of potentials.  One wavenumber
// slot per work item keeps the per-thread state (14 potentials and eight
// packed triangle sums per right-hand side) within the register budget of
// the one-vector kernel; own-domain sources are visited once per slot.

constexpr int NSTAGE_M = 3;

struct __align__(16) StageM {
    float4 pg[TP];           // source points (dx, dy, dz, w), pair-interleaved
    float4 tg[TT];           // triangles (n, h)
    float4 pd[MRG][TP];      // densities of each right-hand side, pair-interleaved
    float4 tc[MRG][2 * TT];  // curl densities of each right-hand side
};
constexpr uint32_t STAGE_M_BYTES = sizeof(StageM);
static_assert(STAGE_M_BYTES == 3584 + MRG * 4096, "multi stage layout");

struct FarSmemM {
    StageM st[NSTAGE_M];
    float4 tab[2 * CHUNK_MAX];
    uint64_t full[NSTAGE_M];
    int cnt[NSTAGE_M];
};

// Per right-hand side: the V and K' sums run packed over the whole item
// (no per-triangle factor; folded once at the end), the K and W terms need
// per-triangle sums (K' and K kept with the sign of -F, as in the one-vector
// kernel).
struct AccM {
    f2 Vr, Vi, nKpr, nKpi;
    float K[2], Wm[2], Wc[6];
};
struct PairTriM {
    f2 nS1r, nS1i, S3r, S3i;
};

template <bool LOSSY>
__device__ __forceinline__ void tile_body_m(const StageM& st, int ntri, int skip_tl, const PairTgt& X, float4 c0,
                                            float Rcf, PairK k, AccM (&acc)[MRG]) {
    const float D2x = c0.x, D2y = c0.y, D2z = c0.z;
    const f2 m2x = bc2(-fmaf(2.f, X.dx, D2x)), m2y = bc2(-fmaf(2.f, X.dy, D2y)), m2z = bc2(-fmaf(2.f, X.dz, D2z));
    const f2 cb = bc2(fmaf(D2x, X.dx, fmaf(D2y, X.dy, fmaf(D2z, X.dz, X.dd))));
    const f2 cn = bc2(fmaf(0.5f, X.nx * D2x + X.ny * D2y + X.nz * D2z, X.nd));
    const f2 Rc2 = bc2(c0.w), Rc = bc2(Rcf);
    const float Xx = fmaf(0.5f, D2x, X.dx), Xy = fmaf(0.5f, D2y, X.dy), Xz = fmaf(0.5f, D2z, X.dz);  // x - c_source
    const f2 z2 = make_float2(0.f, 0.f);
    for (int tl = 0; tl < ntri; tl++) {
        if (tl == skip_tl) continue;  // identical triangle: near-field correction only
        PairTriM S[MRG];
#pragma unroll
        for (int q = 0; q < MRG; q++) S[q] = PairTriM{z2, z2, z2, z2};
        f2 S2r = z2, S2i = z2;
#pragma unroll
        for (int j = 0; j < QP / 2; j++) {
            const float4 GA = st.pg[tl * QP + 2 * j], GB = st.pg[tl * QP + 2 * j + 1];
            const f2 gx = lo2(GA), gy = hi2(GA), gz = lo2(GB), w = hi2(GB);
            const f2 s = fma2(gx, add2(gx, m2x), fma2(gy, add2(gy, m2y), fma2(gz, add2(gz, m2z), cb)));
            const f2 r2 = add2(s, Rc2);
            const f2 rinv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
            const f2 rinv2 = mul2(rinv, rinv);
            const f2 den = fma2(r2, rinv, Rc);  // r + R_c
            const f2 rho = mul2(s, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
            const f2 ndot = fma2(X.nnx, gx, fma2(X.nny, gy, fma2(X.nnz, gz, cn)));
            const f2 arg = fma2(k.kr, rho, k.th);
            f2 sn, cs;
            sincos_approx(arg.x, &sn.x, &cs.x);
            sincos_approx(arg.y, &sn.y, &cs.y);
            f2 a = rinv;
            if constexpr (LOSSY) {
                const f2 e = mul2(k.nkil2, mul2(r2, rinv));
                a = mul2(make_float2(ex2_approx(e.x), ex2_approx(e.y)), rinv);
            }
            const f2 Gr = mul2(a, cs), Gi = mul2(a, sn);
            const f2 B = mul2(k.kr, rinv), nB = mul2(k.nkr, rinv);
            const f2 P = LOSSY ? fma2(k.ki, rinv, rinv2) : rinv2;
            const f2 nFr = fma2(P, Gr, mul2(B, Gi));
            const f2 nFi = fma2(P, Gi, mul2(nB, Gr));
            const f2 nFnr = mul2(ndot, nFr), nFni = mul2(ndot, nFi);
            S2r = fma2(Gr, w, S2r);
            S2i = fma2(Gi, w, S2i);
#pragma unroll
            for (int q = 0; q < MRG; q++) {
                const float4 DA = st.pd[q][tl * QP + 2 * j], DB = st.pd[q][tl * QP + 2 * j + 1];
                const f2 d1r = lo2(DA), d1i = hi2(DA), d2r = lo2(DB), d2i = hi2(DB);
                const f2 nd1i = neg2(d1i), nd2i = neg2(d2i);  // folded into the packed FMAs' operands
                PairTriM& T = S[q];
                AccM& U = acc[q];
                U.Vr = fma2(Gr, d1r, fma2(Gi, nd1i, U.Vr));
                U.Vi = fma2(Gr, d1i, fma2(Gi, d1r, U.Vi));
                U.nKpr = fma2(nFnr, d1r, fma2(nFni, nd1i, U.nKpr));
                U.nKpi = fma2(nFnr, d1i, fma2(nFni, d1r, U.nKpi));
                T.nS1r = fma2(nFr, d2r, fma2(nFi, nd2i, T.nS1r));
                T.nS1i = fma2(nFr, d2i, fma2(nFi, d2r, T.nS1i));
                T.S3r = fma2(Gr, d2r, fma2(Gi, nd2i, T.S3r));
                T.S3i = fma2(Gr, d2i, fma2(Gi, d2r, T.S3i));
            }
        }
        const float4 tg = st.tg[tl];
        const float fK = tg.w - (tg.x * Xx + tg.y * Xy + tg.z * Xz);  // n_t.(y - x)
        const float nn = X.nx * tg.x + X.ny * tg.y + X.nz * tg.z;      // n_x.n_t
        const float s2r = S2r.x + S2r.y, s2i = S2i.x + S2i.y;
#pragma unroll
        for (int q = 0; q < MRG; q++) {
            const PairTriM& T = S[q];
            AccM& t = acc[q];
            const float4 cre = st.tc[q][2 * tl], cim = st.tc[q][2 * tl + 1];
            t.K[0] = fmaf(-fK, T.nS1r.x + T.nS1r.y, t.K[0]);
            t.K[1] = fmaf(-fK, T.nS1i.x + T.nS1i.y, t.K[1]);
            t.Wm[0] = fmaf(nn, T.S3r.x + T.S3r.y, t.Wm[0]);
            t.Wm[1] = fmaf(nn, T.S3i.x + T.S3i.y, t.Wm[1]);
            t.Wc[0] = fmaf(s2r, cre.x, fmaf(-s2i, cim.x, t.Wc[0]));
            t.Wc[1] = fmaf(s2r, cre.y, fmaf(-s2i, cim.y, t.Wc[1]));
            t.Wc[2] = fmaf(s2r, cre.z, fmaf(-s2i, cim.z, t.Wc[2]));
            t.Wc[3] = fmaf(s2r, cim.x, fmaf(s2i, cre.x, t.Wc[3]));
            t.Wc[4] = fmaf(s2r, cim.y, fmaf(s2i, cre.y, t.Wc[4]));
            t.Wc[5] = fmaf(s2r, cim.z, fmaf(s2i, cre.z, t.Wc[5]));
        }
    }
}

// Work item: target tile tx (offset from A.tgt_begin) against source chunk
// cy at wavenumber slot `slot` (0: k0 on every source tile; 1: the target
// domain's k_j on its own tiles), right-hand sides grp * MRG ... + MRG - 1.
template <bool LOSSY>
__device__ __forceinline__ void far32m_item(const FarArgs32M& A, int tx, int cy, int slot, int grp) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FarSmemM& sm = *reinterpret_cast<FarSmemM*>(smem_raw);

    const int tid = threadIdx.x, lane = tid & 31;
    const int tt = A.tgt_begin + tx;
    const int mydom = A.tdom[tt];
    const int2 dr = A.dom_tiles[mydom];
    int sb = A.src_begin + cy * A.chunk_tiles;
    int se = min(sb + A.chunk_tiles, A.src_end);
    if (slot) {
        sb = max(sb, dr.x);
        se = min(se, dr.y);
    }
    const int nsrc = max(0, se - sb);
    const int r0 = grp * MRG;
    const int nq = min(MRG, A.R - r0);

    const int64_t p = (int64_t)tt * TP + tid;
    const float4 g = A.pg[p];
    const int mt = tid / QP;
    const float4 ng = A.tg[(int64_t)tt * TT + mt];
    const double4 ct = A.tc[tt];
    const double2 kk = slot ? A.kdom[mydom] : A.k0;
    const PairK k{bc2((float)kk.x), bc2((float)-kk.x), bc2(0.f), bc2((float)kk.y),
                  bc2((float)(-kk.y * 1.4426950408889634))};
    const PairTgt X{g.x, g.y, g.z, ng.x, ng.y, ng.z, g.x * g.x + g.y * g.y + g.z * g.z,
                    ng.x * g.x + ng.y * g.y + ng.z * g.z, bc2(-ng.x), bc2(-ng.y), bc2(-ng.z)};

    // tile-pair table: 2D, R_c^2, R_c and the FP64-reduced phase
    for (int i = tid; i < nsrc; i += TP) {
        const double4 cs = A.tc[sb + i];
        const double Dx = ct.x - cs.x, Dy = ct.y - cs.y, Dz = ct.z - cs.z;
        const double R = sqrt(Dx * Dx + Dy * Dy + Dz * Dz);
        sm.tab[2 * i] = make_float4((float)(2 * Dx), (float)(2 * Dy), (float)(2 * Dz), (float)(R * R));
        sm.tab[2 * i + 1] = make_float4((float)R, reduce_phase(kk.x * R), 0.f, 0.f);
    }
    if (tid == 0) {
        for (int s = 0; s < NSTAGE_M; s++) {
            mbar_init(&sm.full[s], 1);
            sm.cnt[s] = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int i, int st) {
        const int s = sb + i;
        StageM& S = sm.st[st];
        mbar_arrive_expect_tx(&sm.full[st], STAGE_M_BYTES);
        bulk_g2s(S.pg, A.pgp + (int64_t)s * TP, TP * 16, &sm.full[st]);
        bulk_g2s(S.tg, A.tg + (int64_t)s * TT, TT * 16, &sm.full[st]);
#pragma unroll
        for (int q = 0; q < MRG; q++) {
            const int64_t r = min(r0 + q, A.R - 1);  // a short last group repeats the last vector (not written)
            bulk_g2s(S.pd[q], A.pd + r * A.n_pts + (int64_t)s * TP, TP * 16, &sm.full[st]);
            bulk_g2s(S.tc[q], A.tcurl + r * 2 * A.n_slots + (int64_t)s * 2 * TT, 2 * TT * 16, &sm.full[st]);
        }
    };
    if (tid == 0)
        for (int i = 0; i < min(NSTAGE_M, nsrc); i++) issue(i, i);

    AccM acc[MRG];
#pragma unroll
    for (int q = 0; q < MRG; q++) {
        const f2 z2 = make_float2(0.f, 0.f);
        acc[q].Vr = acc[q].Vi = acc[q].nKpr = acc[q].nKpi = z2;
        acc[q].K[0] = acc[q].K[1] = acc[q].Wm[0] = acc[q].Wm[1] = 0.f;
#pragma unroll
        for (int c = 0; c < 6; c++) acc[q].Wc[c] = 0.f;
    }
    for (int i = 0; i < nsrc; i++) {
        const int st = i % NSTAGE_M;
        mbar_wait_bounded(&sm.full[st], (uint32_t)((i / NSTAGE_M) & 1), A.err);
        const int s = sb + i;
        const int ntri = A.tntri[s];
        const int skip = (s == tt) ? mt : -1;
        const float4 c0 = sm.tab[2 * i], c1 = sm.tab[2 * i + 1];
        PairK kt = k;
        kt.th = bc2(c1.y);
        tile_body_m<LOSSY>(sm.st[st], ntri, skip, X, c0, c1.x, kt, acc);
        // leave the stage; the last warp out refills it with the tile NSTAGE_M ahead
        __syncwarp();
        if (lane == 0) {
            const int old = atomicAdd(&sm.cnt[st], 1);
            if (old == NWARP - 1) {
                sm.cnt[st] = 0;
                if (i + NSTAGE_M < nsrc) issue(i + NSTAGE_M, st);
            }
        }
    }

#pragma unroll
    for (int q = 0; q < MRG; q++) {
        if (q >= nq) break;
        const AccM& t = acc[q];
        // the 14 potentials in the order of the one-vector kernel: PV, PK, PK', PWm, PWc
        const float v[NCOMP] = {t.Vr.x + t.Vr.y, t.Vi.x + t.Vi.y, t.K[0], t.K[1], -(t.nKpr.x + t.nKpr.y),
                                -(t.nKpi.x + t.nKpi.y), t.Wm[0], t.Wm[1], t.Wc[0], t.Wc[1], t.Wc[2], t.Wc[3],
                                t.Wc[4], t.Wc[5]};
        float* out = A.partial + (int64_t)(r0 + q) * A.rstride + ((int64_t)cy * 2 + slot) * NCOMP * A.n_pts + p;
#pragma unroll
        for (int c = 0; c < NCOMP; c++) out[(int64_t)c * A.n_pts] = v[c];
    }
}

__global__ void __launch_bounds__(TP, 2) far32m_kernel(FarArgs32M A) {
    const int4 w = A.work[blockIdx.x];
    const int mydom = A.tdom[A.tgt_begin + w.x];
    const double ki = w.z ? A.kdom[mydom].y : A.k0.y;
    if (ki != 0.0) far32m_item<true>(A, w.x, w.y, w.z, w.w);
    else far32m_item<false>(A, w.x, w.y, w.z, w.w);
}

cudaError_t launch_far32_multi(const FarArgs32M& a, int64_t n_work, cudaStream_t s) {
    const size_t smem = sizeof(FarSmemM);
    static const cudaError_t attr_e =
        cudaFuncSetAttribute(far32m_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr_e != cudaSuccess) return attr_e;
    if (n_work <= 0) return cudaSuccess;
    far32m_kernel<<<(unsigned)n_work, TP, smem, s>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- FP64 far field

// One vector at FP64: the multi-vector kernel with a single group.
cudaError_t launch_far64(const FarArgs64& a, int n_tgt_tiles, int n_chunks, cudaStream_t s) {
    FarArgs64M m{};
    m.pg = a.pg; m.tg = a.tg; m.tc = a.tc; m.tdom = a.tdom; m.tntri = a.tntri; m.pd = a.pd; m.tcurl = a.tcurl;
    m.dom_tiles = a.dom_tiles; m.kdom = a.kdom; m.k0 = a.k0;
    m.src_begin = a.src_begin; m.src_end = a.src_end; m.tgt_begin = a.tgt_begin; m.chunk_tiles = a.chunk_tiles;
    m.slot1 = a.slot1; m.groups = 1; m.R = 1; m.n_pts = a.n_pts; m.n_slots = 0; m.rstride = 0; m.partial = a.partial;
    return launch_far64_multi(m, n_tgt_tiles, n_chunks, s);
}

// Several vectors per FP64 far-field CTA.  The Green's function G, its radial
// factor F and the geometric weights of a (target point, source point) pair
// are computed once and applied to each of the group's vectors, with the
// target-normal and source-edge factors folded into the point terms:
// 16 FP64 FMAs per vector and pair beside the shared evaluation (sqrt, the
// reciprocal, sincos and, for a complex wavenumber, exp).  Sums per vector
// and component in source order, so results do not depend on the group.
template <int RG, bool ATTEN>
__device__ __forceinline__ void far64m_body(const FarArgs64M& A, int sl, int grp) {
    const int tid = threadIdx.x;
    const int tt = A.tgt_begin + blockIdx.x;
    const int chunk = blockIdx.y;
    int sb = A.src_begin + chunk * A.chunk_tiles;
    int se = min(sb + A.chunk_tiles, A.src_end);
    const int64_t p = (int64_t)tt * TP + tid;
    const double4 g = A.pg[p];
    const int mt = tid / QP;
    const double4 ng = A.tg[(int64_t)tt * TT + mt];
    const double4 ct = A.tc[tt];
    const int mydom = A.tdom[tt];
    if (sl == 1) {
        const int2 dr = A.dom_tiles[mydom];
        sb = max(sb, dr.x);
        se = min(se, dr.y);
    }
    const double2 kk = sl ? A.kdom[mydom] : A.k0;
    const double kr = kk.x, ki = kk.y;
    const int r0 = grp * RG, nv = min(RG, A.R - r0);
    double acc[RG][NCOMP];
#pragma unroll
    for (int v = 0; v < RG; v++)
#pragma unroll
        for (int c = 0; c < NCOMP; c++) acc[v][c] = 0.0;
    for (int s = sb; s < se; s++) {
        const double4 cs = A.tc[s];
        const double Xx = g.x + (ct.x - cs.x), Xy = g.y + (ct.y - cs.y), Xz = g.z + (ct.z - cs.z);  // x - c_source
        const int ntri = A.tntri[s];
        for (int tl = 0; tl < ntri; tl++) {
            if (s == tt && tl == mt) continue;
            const int64_t ts = (int64_t)s * TT + tl;
            const double4 tg = A.tg[ts];
            const double fK = tg.w - (tg.x * Xx + tg.y * Xy + tg.z * Xz);
            const double nn = ng.x * tg.x + ng.y * tg.y + ng.z * tg.z;
            double S2r = 0, S2i = 0;
            for (int q = 0; q < QP; q++) {
                const double4 y = A.pg[ts * QP + q];
                const double ex = Xx - y.x, ey = Xy - y.y, ez = Xz - y.z;  // x - y
                const double r = sqrt(ex * ex + ey * ey + ez * ez);
                const double rinv = 1.0 / r;
                double sn, cs2;
                sincos(kr * r, &sn, &cs2);
                const double a = (ATTEN ? exp(-ki * r) : 1.0) * rinv;
                const double Gr = a * cs2, Gi = a * sn;
                const double u = -ki - rinv;
                const double Fr = (Gr * u - Gi * kr) * rinv, Fi = (Gr * kr + Gi * u) * rinv;
                const double ndot = ng.x * ex + ng.y * ey + ng.z * ez;
                const double nFr = ndot * Fr, nFi = ndot * Fi;  // K' point factor
                const double kFr = fK * Fr, kFi = fK * Fi;      // K point factor
                const double wGr = nn * Gr, wGi = nn * Gi;      // W (normal-normal) point factor
                S2r += Gr * y.w;
                S2i += Gi * y.w;
#pragma unroll
                for (int v = 0; v < RG; v++) {
                    if (v >= nv) break;
                    const double4 d = A.pd[(int64_t)(r0 + v) * A.n_pts + ts * QP + q];
                    acc[v][0] += Gr * d.x - Gi * d.y;
                    acc[v][1] += Gr * d.y + Gi * d.x;
                    acc[v][2] += kFr * d.z - kFi * d.w;
                    acc[v][3] += kFr * d.w + kFi * d.z;
                    acc[v][4] += nFr * d.x - nFi * d.y;
                    acc[v][5] += nFr * d.y + nFi * d.x;
                    acc[v][6] += wGr * d.z - wGi * d.w;
                    acc[v][7] += wGr * d.w + wGi * d.z;
                }
            }
#pragma unroll
            for (int v = 0; v < RG; v++) {
                if (v >= nv) break;
                const double4* tcv = A.tcurl + (int64_t)(r0 + v) * 2 * A.n_slots;
                const double4 cre = tcv[2 * ts], cim = tcv[2 * ts + 1];
                acc[v][8] += S2r * cre.x - S2i * cim.x;
                acc[v][9] += S2r * cre.y - S2i * cim.y;
                acc[v][10] += S2r * cre.z - S2i * cim.z;
                acc[v][11] += S2r * cim.x + S2i * cre.x;
                acc[v][12] += S2r * cim.y + S2i * cre.y;
                acc[v][13] += S2r * cim.z + S2i * cre.z;
            }
        }
    }
#pragma unroll
    for (int v = 0; v < RG; v++) {
        if (v >= nv) break;
        double* out = A.partial + (int64_t)(r0 + v) * A.rstride + ((int64_t)chunk * 2 + sl) * NCOMP * A.n_pts + p;
#pragma unroll
        for (int c = 0; c < NCOMP; c++) out[(int64_t)c * A.n_pts] = acc[v][c];
    }
}

template <int RG>
__global__ void __launch_bounds__(TP, RG == 1 ? 2 : 1) far64m_kernel(FarArgs64M A) {
    const int sl = blockIdx.z / A.groups, grp = blockIdx.z % A.groups;
    const double ki = sl ? A.kdom[A.tdom[A.tgt_begin + blockIdx.x]].y : A.k0.y;
    if (ki != 0.0) far64m_body<RG, true>(A, sl, grp);
    else far64m_body<RG, false>(A, sl, grp);
}

// One vector (groups = R = 1) or groups of RG64; slot 1 only with a.slot1.
cudaError_t launch_far64_multi(const FarArgs64M& a, int n_tgt_tiles, int n_chunks, cudaStream_t s) {
    if (n_tgt_tiles <= 0 || n_chunks <= 0 || a.groups <= 0) return cudaSuccess;
    const dim3 grid(n_tgt_tiles, n_chunks, (a.slot1 ? 2 : 1) * a.groups);
    if (a.R == 1) far64m_kernel<1><<<grid, TP, 0, s>>>(a);
    else far64m_kernel<RG64><<<grid, TP, 0, s>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- projection onto P1 test functions

// One CTA per target tile.  Its TP threads first sum, each for its own
// point, the chunk partials of both slots (reads coalesced across the CTA);
// then one thread per triangle projects onto the P1 test functions from
// shared memory.  FP32 partials are summed with a compensated (TwoSum)
// FP32 sum in chunk order, converted to FP64 once: the GPU's FP64 rate is
// a small fraction of its FP32 rate, and the compensation carries the
// rounding error of every addition, so the result matches an FP64 sum of
// the same FP32 values to about 1e-15 of the sum of their magnitudes.
__global__ void __launch_bounds__(TP) project_kernel(ProjectArgs a) {
    __shared__ double Ps[2][NCOMP][TP];
    const int tile = a.tgt_begin + blockIdx.x;
    const int tid = threadIdx.x;
    const int tdom = a.tdom[tile];
    {
        const int64_t p = (int64_t)tile * TP + tid;
        for (int sl = 0; sl < 2; sl++) {
            const SlotCoef cf = a.coef[tdom * 2 + sl];
            if (cf.cV == 0 && cf.cK == 0 && cf.cKp == 0 && cf.cW == 0) continue;
            const int64_t step = 2 * NCOMP * a.n_pts;  // one chunk
            if (a.partial32) {
                // all components at once: NCOMP independent loads per chunk
                const float* src = a.partial32 + (int64_t)sl * NCOMP * a.n_pts + (p - a.p_off);
                float hi[NCOMP], lo[NCOMP];
#pragma unroll
                for (int c = 0; c < NCOMP; c++) hi[c] = lo[c] = 0.f;
                for (int ch = 0; ch < a.n_chunks; ch++, src += step) {
                    float x[NCOMP];
#pragma unroll
                    for (int c = 0; c < NCOMP; c++) x[c] = src[(int64_t)c * a.n_pts];
#pragma unroll
                    for (int c = 0; c < NCOMP; c++) {
                        const float u = hi[c] + x[c];  // TwoSum: hi + x = u + (rounding error)
                        const float xb = u - hi[c];
                        lo[c] += (hi[c] - (u - xb)) + (x[c] - xb);
                        hi[c] = u;
                    }
                }
#pragma unroll
                for (int c = 0; c < NCOMP; c++) Ps[sl][c][tid] = (double)hi[c] + (double)lo[c];
            } else {
                for (int c = 0; c < NCOMP; c++) {
                    const double* src = a.partial64 + ((int64_t)sl * NCOMP + c) * a.n_pts + (p - a.p_off);
                    double sum = 0.0;
                    for (int ch = 0; ch < a.n_chunks; ch++) sum += src[ch * step];
                    Ps[sl][c][tid] = sum;
                }
            }
        }
    }
    __syncthreads();
    // far part: thread tid < TT owns slot tile * TT + tid
    const int64_t s = (int64_t)tile * TT + tid;
    const bool own = tid < TT && a.slot_v[s].x >= 0;
    double r1[3][2] = {{0, 0}, {0, 0}, {0, 0}}, r2[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    if (own) {
        const int dom = tdom;  // a tile holds triangles of one domain
        const double inv4pi = 0.07957747154594767;
        for (int sl = 0; sl < 2; sl++) {
            const SlotCoef cf = a.coef[dom * 2 + sl];
            if (cf.cV == 0 && cf.cK == 0 && cf.cKp == 0 && cf.cW == 0) continue;
            double wc[6] = {0, 0, 0, 0, 0, 0};
            for (int q = 0; q < QP; q++) {
                const int64_t p = s * QP + q;
                double P[NCOMP];
                for (int c = 0; c < NCOMP; c++) P[c] = Ps[sl][c][tid * QP + q];
                const double w = a.pt_w[p] * inv4pi;
                // row1 potential: cV PV - cK PK ; row2 (pointwise part): cKp PKp - cW k^2 PWm
                const double t1r = cf.cV * P[0] - cf.cK * P[2], t1i = cf.cV * P[1] - cf.cK * P[3];
                const double kwr = cf.k2re * P[6] - cf.k2im * P[7], kwi = cf.k2re * P[7] + cf.k2im * P[6];
                const double t2r = cf.cKp * P[4] - cf.cW * kwr, t2i = cf.cKp * P[5] - cf.cW * kwi;
                for (int k = 0; k < 3; k++) {
                    const double wl = w * a.lam[q][k];
                    r1[k][0] += wl * t1r;
                    r1[k][1] += wl * t1i;
                    r2[k][0] += wl * t2r;
                    r2[k][1] += wl * t2i;
                }
                for (int c = 0; c < 6; c++) wc[c] += w * P[8 + c];
            }
            for (int k = 0; k < 3; k++) {
                const double* cu = &a.slot_curl[s * 9 + 3 * k];
                r2[k][0] += cf.cW * (cu[0] * wc[0] + cu[1] * wc[1] + cu[2] * wc[2]);
                r2[k][1] += cf.cW * (cu[0] * wc[3] + cu[1] * wc[4] + cu[2] * wc[5]);
            }
        }
    }
    // near pairs (touching and near band): combined 3x3 sub-blocks (row1<-psi,
    // row1<-phi, row2<-psi, row2<-phi).  Every thread takes part: thread
    // (j, sub) = (tid / NSUB, tid % NSUB) sums every NSUB-th pair of slot
    // tile * TT + j; the NSUB partial sums meet in shared memory (Ps is free
    // again) and are added in a fixed order, so results are deterministic.
    // FP32 blocks (the FP32 operator) take FP32 products and sums.
    if (a.np_ptr) {
        constexpr int NSUB = TP / TT;
        double* red = &Ps[0][0][0];  // [TT][NSUB][12]
        static_assert(TT * NSUB * 12 <= 2 * NCOMP * TP, "near partial sums fit in the potential buffer");
        __syncthreads();
        const int j = tid / NSUB, sub = tid % NSUB;
        const int64_t sj = (int64_t)tile * TT + j;
        double acc[12];
#pragma unroll
        for (int c = 0; c < 12; c++) acc[c] = 0;
        if (a.slot_v[sj].x >= 0) {
            const int64_t pe = a.np_ptr[sj + 1];
            if (a.nb32) {
                float f[12];
#pragma unroll
                for (int c = 0; c < 12; c++) f[c] = 0.f;
                for (int64_t pi = a.np_ptr[sj] + sub; pi < pe; pi += NSUB) {
                    const int4 vt = a.slot_v[a.np_src[pi]];
                    const int vid[3] = {vt.x, vt.y, vt.z};
                    float2 xv[2][3];
#pragma unroll
                    for (int b = 0; b < 3; b++) {
                        const double2 x1 = a.x[a.v_dof1[vid[b]]], x2 = a.x[a.v_dof2[vid[b]]];
                        xv[0][b] = make_float2((float)x1.x, (float)x1.y);
                        xv[1][b] = make_float2((float)x2.x, (float)x2.y);
                    }
                    // 36 complex entries as 18 aligned float4 (pair stride 288 bytes)
                    const float4* B4 = reinterpret_cast<const float4*>(a.nb32 + pi * 36);
#pragma unroll
                    for (int e2 = 0; e2 < 18; e2++) {
                        const float4 B = B4[e2];
#pragma unroll
                        for (int h = 0; h < 2; h++) {
                            const int e = 2 * e2 + h, blk = e / 9, k = (e % 9) / 3, b = e % 3;
                            const float br = h ? B.z : B.x, bi = h ? B.w : B.y;
                            const float2 x = xv[blk & 1][b];
                            const int o = (blk < 2 ? 0 : 6) + 2 * k;
                            f[o] = fmaf(br, x.x, fmaf(-bi, x.y, f[o]));
                            f[o + 1] = fmaf(br, x.y, fmaf(bi, x.x, f[o + 1]));
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < 12; c++) acc[c] = f[c];
            } else {
                for (int64_t pi = a.np_ptr[sj] + sub; pi < pe; pi += NSUB) {
                    const int4 vt = a.slot_v[a.np_src[pi]];
                    const int vid[3] = {vt.x, vt.y, vt.z};
                    double2 xv[2][3];
                    for (int b = 0; b < 3; b++) {
                        xv[0][b] = a.x[a.v_dof1[vid[b]]];
                        xv[1][b] = a.x[a.v_dof2[vid[b]]];
                    }
#pragma unroll
                    for (int e = 0; e < 36; e++) {
                        const int blk = e / 9, k = (e % 9) / 3, b = e % 3;
                        const double2 B = a.nb64[pi * 36 + e];
                        const double2 x = xv[blk & 1][b];
                        const int o = (blk < 2 ? 0 : 6) + 2 * k;
                        acc[o] += B.x * x.x - B.y * x.y;
                        acc[o + 1] += B.x * x.y + B.y * x.x;
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 12; c++) red[(j * NSUB + sub) * 12 + c] = acc[c];
        __syncthreads();
        if (own)
            for (int u = 0; u < NSUB; u++) {
                const double* q = red + (tid * NSUB + u) * 12;
                for (int k = 0; k < 3; k++) {
                    r1[k][0] += q[2 * k];
                    r1[k][1] += q[2 * k + 1];
                    r2[k][0] += q[6 + 2 * k];
                    r2[k][1] += q[6 + 2 * k + 1];
                }
            }
    }
    if (!own) return;
    for (int k = 0; k < 3; k++) {
        a.tri_out[(s * 3 + k) * 2] = make_double2(r1[k][0], r1[k][1]);
        a.tri_out[(s * 3 + k) * 2 + 1] = make_double2(r2[k][0], r2[k][1]);
    }
}

cudaError_t launch_project(const ProjectArgs& a, cudaStream_t s) {
    const int n_tiles = a.tgt_end - a.tgt_begin;
    if (n_tiles <= 0) return cudaSuccess;
    project_kernel<<<(unsigned)n_tiles, TP, 0, s>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- vertex reduction

__global__ void reduce_kernel(ReduceArgs a) {
    const int64_t v = a.v_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.v_end) return;
    double s1r = 0, s1i = 0, s2r = 0, s2i = 0;
    for (int64_t i = a.vc_ptr[v]; i < a.vc_ptr[v + 1]; i++) {
        const int64_t c = a.vc_idx[i];
        const double2 u = a.tri_out[c * 2], w = a.tri_out[c * 2 + 1];
        s1r += u.x;
        s1i += u.y;
        s2r += w.x;
        s2i += w.y;
    }
    a.y[a.v_dof1[v]] = make_double2(s1r, s1i);
    a.y[a.v_dof2[v]] = make_double2(s2r, s2i);
}

cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t s) {
    int64_t n = a.v_end - a.v_begin;
    if (n <= 0) return cudaSuccess;
    reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s) {
    int64_t n = a.s_end - a.s_begin;
    if (n <= 0) return cudaSuccess;
    gather_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gbem
