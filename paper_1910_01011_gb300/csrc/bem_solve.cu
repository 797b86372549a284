// bem_solve.cu -- incident fields and right-hand sides (paper Sec. 2.3 eq.
// Galerkin_disc_rhs1: b_r = <gamma^{j,+} p_inc, eta_r>), with the same
// regular rule as the operator.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include <algorithm>
#include <chrono>
#include <complex>
#include <vector>

#include "ctx.h"
#include "df_math.cuh"
#include "internal.h"
#include "krylov.h"

using namespace gbem;

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

namespace gbem {

struct PlaneWaveArgs {
    const double4* pg;   // (dx, dy, dz, w)
    const double4* tc;
    const int4* slot_v;
    const double* slot_n;
    double d[3];
    double2 amp, k0;
    int64_t n_slots;
    double lam[QP][3];
    double2* tri_out;
};

// Per slot: <p_inc, phi_k> and <dp_inc/dn, phi_k> on the triangle with the
// regular rule; p_inc = amp exp(i k0 d.x), dp/dn = i k0 (d.n) p_inc.
__global__ void plane_wave_kernel(PlaneWaveArgs a) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n_slots) return;
    if (a.slot_v[s].x < 0) return;
    const double4 c = a.tc[s / TT];
    const double dn = a.d[0] * a.slot_n[3 * s] + a.d[1] * a.slot_n[3 * s + 1] + a.d[2] * a.slot_n[3 * s + 2];
    double r[3][2][2] = {};
    for (int q = 0; q < QP; q++) {
        const double4 g = a.pg[s * QP + q];
        const double x = c.x + g.x, y = c.y + g.y, z = c.z + g.z;
        const double ph = a.d[0] * x + a.d[1] * y + a.d[2] * z;
        // exp(i k0 ph) with complex k0
        double sn, cs;
        sincos(a.k0.x * ph, &sn, &cs);
        const double m = exp(-a.k0.y * ph);
        const double er = m * cs, ei = m * sn;
        const double pr = a.amp.x * er - a.amp.y * ei, pi = a.amp.x * ei + a.amp.y * er;
        // i k0 dn p
        const double kr = -a.k0.y * dn, ki = a.k0.x * dn;
        const double qr = kr * pr - ki * pi, qi = kr * pi + ki * pr;
        for (int k = 0; k < 3; k++) {
            const double wl = g.w * a.lam[q][k];
            r[k][0][0] += wl * pr;
            r[k][0][1] += wl * pi;
            r[k][1][0] += wl * qr;
            r[k][1][1] += wl * qi;
        }
    }
    for (int k = 0; k < 3; k++) {
        a.tri_out[(s * 3 + k) * 2] = make_double2(r[k][0][0], r[k][0][1]);
        a.tri_out[(s * 3 + k) * 2 + 1] = make_double2(r[k][1][0], r[k][1][1]);
    }
}

struct PistonArgs {
    const double4* pg;   // (dx, dy, dz, w)
    const double4* tc;
    const int4* slot_v;
    const double* slot_n;
    const float4 *disc_h, *disc_l;  // [n_elem * nq] (x, y, z, weight) as double-floats
    int n_elem, nq;
    const float4* w;     // [n_rhs][n_elem] piston weights (re hi, re lo, im hi, im lo)
    int n_rhs;
    float4 k0;           // (Re hi, lo, Im hi, lo)
    double2 pref;        // -i omega rho0 / (2 pi)
    int64_t n_slots;
    double lam[QP][3];
    DfConsts c;
    const float4* sctab; // double-float sin / cos table (df_math.cuh)
    const float2* extab;
    double2* tri_out;    // [n_rhs][n_slots*3][2]
};

// Excitations per block row of piston_kernel (its accumulators live in
// registers: 4 double-floats per excitation and thread).
constexpr int PK_RC = 16;
constexpr int PK_SLOTS = 16;  // slots per block; one thread per (slot, rule point)

__device__ __forceinline__ void dacc(dfl& acc, dfl x) {  // acc += x (low part gathers the errors)
    const dfl q = two_sum(acc.h, x.h);
    acc.h = q.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(q.l, x.l));
}

// Rayleigh field of piston m (its disc points, weights folded in) at x and
// its normal derivative along n, in double-float arithmetic:
// e = sum_j w_j exp(ik R_j)/R_j, f = sum_j w_j exp(ik R_j)/R_j (ik - 1/R_j) (x - y_j).n / R_j.
template <bool ATTEN>
__device__ __forceinline__ void piston_field(const PistonArgs& a, int m, const dfl (&x)[3], const dfl (&n)[3],
                                             const float4* __restrict__ tab, const float2* __restrict__ etab,
                                             dfl& er, dfl& ei, dfl& fr, dfl& fi) {
    const dfl kr = {a.k0.x, a.k0.y}, ki = {a.k0.z, a.k0.w};
    er = ei = fr = fi = dfl{0.0f, 0.0f};
    for (int j = 0; j < a.nq; j++) {
        const float4 dh = a.disc_h[(int64_t)m * a.nq + j], dl = a.disc_l[(int64_t)m * a.nq + j];
        const dfl ex = dsub(x[0], dfl{dh.x, dl.x}), ey = dsub(x[1], dfl{dh.y, dl.y}), ez = dsub(x[2], dfl{dh.z, dl.z});
        dfl R, Ri;
        dsqrt_rinv(dadd(dadd(dsqr(ex), dsqr(ey)), dsqr(ez)), R, Ri);
        dfl sn, cs;
        dsincos(dmul(kr, R), a.c, tab, sn, cs);
        dfl amp = dmul(Ri, dfl{dh.w, dl.w});
        if (ATTEN) amp = dmul(amp, dexp_neg(dmul(ki, R), a.c, etab));
        const dfl gr = dmul(amp, cs), gi = dmul(amp, sn);  // w exp(ikR)/R
        dacc(er, gr);
        dacc(ei, gi);
        // d/dn: exp(ikR)/R (ik - 1/R) (x-y).n / R
        const dfl ur = dsub(dneg(ki), Ri);
        const dfl dn = dmul(dadd(dadd(dmul(ex, n[0]), dmul(ey, n[1])), dmul(ez, n[2])), Ri);
        dacc(fr, dmul(dsub(dmul(gr, ur), dmul(gi, kr)), dn));
        dacc(fi, dmul(dadd(dmul(gr, kr), dmul(gi, ur)), dn));
    }
}

// Per slot and excitation: <p_inc, phi_k> and <dp_inc/dn, phi_k> with the
// Rayleigh sum over piston discs (baffled-piston reading of the transducer
// field; the paper defers it to its ref. elwin2015, Sec. 3.2).  The Green's
// function sums do not depend on the weights, so each thread evaluates every
// piston's field once at its rule point and accumulates it into the PK_RC
// excitations of its block row; a piston whose weight is zero in all of them
// is skipped (a block-uniform test), so the unit excitations of a
// superposition basis cost one evaluation per piston.  The sums run in
// double-float FP32 arithmetic (df_math.cuh: FP64 accuracy at the FP32
// rate); the rule points of a slot are summed against the P1 values in
// shared memory in FP64.
template <bool ATTEN>
__global__ void __launch_bounds__(PK_SLOTS * QP) piston_kernel(PistonArgs a) {
    __shared__ float4 tab[128];
    __shared__ float2 etab[64];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) tab[i] = a.sctab[i];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) etab[i] = a.extab[i];
    __syncthreads();
    const int sl = threadIdx.x / QP, q = threadIdx.x % QP;
    const int64_t s = (int64_t)blockIdx.x * PK_SLOTS + sl;
    const int r0 = blockIdx.y * PK_RC, nrc = min(PK_RC, a.n_rhs - r0);
    const bool live = s < a.n_slots && a.slot_v[s].x >= 0;
    dfl acc[PK_RC][4];
#pragma unroll
    for (int c = 0; c < PK_RC; c++) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = dfl{0.0f, 0.0f};
    double gw = 0;
    if (live) {
        const double4 c0 = a.tc[s / TT];
        const double4 g = a.pg[s * QP + q];
        gw = g.w;
        const double xd[3] = {c0.x + g.x, c0.y + g.y, c0.z + g.z};
        dfl x[3], n[3];
        for (int k = 0; k < 3; k++) {
            const float h = (float)xd[k];
            x[k] = dfl{h, (float)(xd[k] - (double)h)};
            const double nd = a.slot_n[3 * s + k];
            const float nh = (float)nd;
            n[k] = dfl{nh, (float)(nd - (double)nh)};
        }
        const float4* wr = a.w + (int64_t)r0 * a.n_elem;
        for (int m = 0; m < a.n_elem; m++) {
            bool any = false;
            for (int c = 0; c < nrc && !any; c++) {
                const float4 wm = wr[(int64_t)c * a.n_elem + m];
                any = wm.x != 0.0f || wm.z != 0.0f;
            }
            if (!any) continue;
            dfl er, ei, fr, fi;
            piston_field<ATTEN>(a, m, x, n, tab, etab, er, ei, fr, fi);
#pragma unroll
            for (int c = 0; c < PK_RC; c++)
                if (c < nrc) {
                    const float4 wm = wr[(int64_t)c * a.n_elem + m];
                    const dfl wre = {wm.x, wm.y}, wim = {wm.z, wm.w};
                    dmac(acc[c][0], wre, er, 1.0f);
                    dmac(acc[c][0], wim, ei, -1.0f);
                    dmac(acc[c][1], wre, ei, 1.0f);
                    dmac(acc[c][1], wim, er, 1.0f);
                    dmac(acc[c][2], wre, fr, 1.0f);
                    dmac(acc[c][2], wim, fi, -1.0f);
                    dmac(acc[c][3], wre, fi, 1.0f);
                    dmac(acc[c][3], wim, fr, 1.0f);
                }
        }
    }
    // Galerkin moments out_k = sum_q w_q lam_qk (pref x) in rule order; after
    // the exchange, thread (sl, q) writes trace q & 1 of P1 function q >> 1
    __shared__ double sh[PK_SLOTS][QP][5];
    static_assert(QP == 6, "one output (3 P1 functions x 2 traces) per rule point");
    const int k = q >> 1, tr = q & 1;
#pragma unroll
    for (int c = 0; c < PK_RC; c++) {
        if (c >= nrc) break;
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = (double)acc[c][u].h + (double)acc[c][u].l;
        sh[sl][q][0] = a.pref.x * v[0] - a.pref.y * v[1];
        sh[sl][q][1] = a.pref.x * v[1] + a.pref.y * v[0];
        sh[sl][q][2] = a.pref.x * v[2] - a.pref.y * v[3];
        sh[sl][q][3] = a.pref.x * v[3] + a.pref.y * v[2];
        sh[sl][q][4] = gw;
        __syncthreads();
        if (live) {
            double vr = 0, vi = 0;
            for (int qq = 0; qq < QP; qq++) {
                const double wl = sh[sl][qq][4] * a.lam[qq][k];
                vr += wl * sh[sl][qq][2 * tr];
                vi += wl * sh[sl][qq][2 * tr + 1];
            }
            a.tri_out[(int64_t)(r0 + c) * a.n_slots * 6 + (s * 3 + k) * 2 + tr] = make_double2(vr, vi);
        }
        __syncthreads();
    }
}

constexpr int64_t BLOCK_COLS = 16;  // widest block of block GMRES

int64_t solve_batch_width(const bem_solve_opts& o, int64_t n_exc) {
    const int64_t lead = std::max<int64_t>(1, std::min<int64_t>(o.batch_rhs, n_exc));
    if (!o.block_gmres) return lead;
    const int64_t groups = (lead + BLOCK_COLS - 1) / BLOCK_COLS;
    return (lead + groups - 1) / groups;
}

struct SolveState {
    Krylov kry;
    double2* b = nullptr;       // [n_rhs][N]
    double2* u = nullptr;       // [n_rhs][N] solutions
    double2* r = nullptr;       // work
    double2* d = nullptr;       // work
    double2* pb = nullptr;      // work
    // batched solves: [batch][N] work blocks
    double2 *bt = nullptr, *bpb = nullptr, *bd = nullptr, *br = nullptr;
    int64_t batch_alloc = 0;
    double2* tri_rhs = nullptr; // [n_rhs][n_slots*6]
    double4* disc = nullptr;    // piston disc points [n_elem * nq] (x, y, z, weight)
    double2* wdev = nullptr;    // piston weights [n_rhs][n_elem]
    float4* disc_df = nullptr;  // the same as double-floats: [2][n_elem * nq] (hi, lo)
    float4* w_df = nullptr;     // [n_rhs][n_elem] (re hi, re lo, im hi, im lo)
    int64_t n_rhs_alloc = 0;
    int64_t n_rhs_solved = 0;
    // superposition basis: the solution of every piston alone, [n_elem][N]
    double2* basis = nullptr;
    int64_t n_basis = 0;
    double2* wstage = nullptr;  // staging for superposition weights and outputs
    size_t wstage_bytes = 0;
    // recycled solution space (bem_solve_opts.recycle): Q [rec_cap][N] orthonormal
    // right-hand sides of earlier solves, U [rec_cap][N] with A_hat U = Q, rec_k in use
    double2 *rec_Q = nullptr, *rec_U = nullptr, *rec_C = nullptr;  // rec_C: [rec_cap][REC_RMAX] coefficients
    int64_t rec_cap = 0, rec_k = 0;
};

constexpr int REC_RMAX = 64;  // columns per coefficient pass of the recycled space

// C[k][r] = sum_i conj(Q_k[i]) B_r[i] (k < gridDim.x, r < gridDim.y; row stride REC_RMAX)
__global__ void rec_dots_kernel(const double2* __restrict__ Q, const double2* __restrict__ B, int64_t N,
                                double2* __restrict__ C) {
    const int k = blockIdx.x, r = blockIdx.y;
    const double2* q = Q + (int64_t)k * N;
    const double2* b = B + (int64_t)r * N;
    double sr = 0, si = 0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double2 a = q[i], x = b[i];
        sr += a.x * x.x + a.y * x.y;
        si += a.x * x.y - a.y * x.x;
    }
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][w] = sr;
        red[1][w] = si;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0, ti = 0;
        for (int j = 0; j < (int)(blockDim.x >> 5); j++) {
            tr += red[0][j];
            ti += red[1][j];
        }
        C[(int64_t)k * REC_RMAX + r] = make_double2(tr, ti);
    }
}

// X_r[i] = base_r[i] + alpha sum_{k < K} U_k[i] C[k][r]   (base may be null)
__global__ void rec_combine_kernel(const double2* __restrict__ U, int K, const double2* __restrict__ C, int64_t N,
                                   double alpha, const double2* base, double2* X) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= N) return;
    double xr = 0, xi = 0;
    for (int k = 0; k < K; k++) {
        const double2 a = U[(int64_t)k * N + i], c = C[(int64_t)k * REC_RMAX + r];
        xr += a.x * c.x - a.y * c.y;
        xi += a.x * c.y + a.y * c.x;
    }
    double2 v = base ? base[(int64_t)r * N + i] : make_double2(0, 0);
    v.x += alpha * xr;
    v.y += alpha * xi;
    X[(int64_t)r * N + i] = v;
}

__global__ void rec_scale_kernel(const double2* __restrict__ x, int64_t N, double s, double2* __restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[i] = make_double2(s * x[i].x, s * x[i].y);
}

}  // namespace gbem

// Right-hand sides of every excitation into S->b (device).
// r0 > 0 (excitations joined to a running solve): only excitations
// [r0, r0 + count) are built, into storage already sized (capacity) by the
// first call; the piston discs of that call are reused.
static int build_rhs(bem_ctx* ctx, int64_t r0 = 0, int64_t count = -1, int64_t capacity = 0) {
    const Geometry& g = ctx->geo;
    SolveState* S = ctx->solve;
    const int64_t N = g.n_dof, nr = ctx->field_kind == 2 ? ctx->n_rhs : 1;
    if (count < 0) count = nr - r0;
    int rc;
    if (r0 > 0 && (ctx->field_kind != 2 || S->n_rhs_alloc < r0 + count || !S->disc_df))
        return ctx->fail(BEM_ERR_STATE, "joined excitations beyond the solve's capacity");
    if (S->n_rhs_alloc < std::max(nr, capacity)) {
        const int64_t cap = std::max(nr, capacity);
        for (void* p : {(void*)S->b, (void*)S->u, (void*)S->tri_rhs}) ctx->dfree(p);
        S->b = (double2*)ctx->dalloc(cap * N * sizeof(double2), &rc); if (rc) return rc;
        S->u = (double2*)ctx->dalloc(cap * N * sizeof(double2), &rc); if (rc) return rc;
        S->tri_rhs = (double2*)ctx->dalloc(cap * g.n_slots * 6 * sizeof(double2), &rc); if (rc) return rc;
        S->n_rhs_alloc = cap;
    }
    if (ctx->field_kind == 1) {
        PlaneWaveArgs a{};
        a.pg = ctx->dev.pg64; a.tc = ctx->dev.tc; a.slot_v = ctx->dev.slot_v; a.slot_n = ctx->dev.slot_n;
        for (int i = 0; i < 3; i++) a.d[i] = ctx->pw_dir[i];
        a.amp = make_double2(ctx->pw_amp[0], ctx->pw_amp[1]);
        a.k0 = make_double2(ctx->k0re, ctx->k0im);
        a.n_slots = g.n_slots;
        for (int q = 0; q < QP; q++)
            for (int k = 0; k < 3; k++) a.lam[q][k] = ctx->quad.lam[q][k];
        a.tri_out = S->tri_rhs;
        CK(cudaMemsetAsync(S->tri_rhs, 0, g.n_slots * 6 * sizeof(double2), ctx->stream));
        plane_wave_kernel<<<(unsigned)((g.n_slots + 127) / 128), 128, 0, ctx->stream>>>(a);
        ctx->launches++;
    } else if (ctx->field_kind == 2) {
        // piston disc points: n_r Gauss radii x n_t angles per piston
        const int n_r = 4, n_t = 8, nq = n_r * n_t;
        const int64_t ne = (int64_t)ctx->tr_r.size();
        std::vector<double> gx, gw;
        gauss_legendre01(n_r, gx, gw);
        std::vector<double4> disc(r0 > 0 ? 0 : ne * nq);
        for (int64_t m = 0; m < (r0 > 0 ? 0 : ne); m++) {
            const double* c = &ctx->tr_c[3 * m];
            const double* nn = &ctx->tr_n[3 * m];
            const double a = ctx->tr_r[m];
            const double ax[3] = {std::fabs(nn[2]) > 0.9 ? 1.0 : 0.0, 0.0, std::fabs(nn[2]) > 0.9 ? 0.0 : 1.0};
            double e1[3] = {ax[1] * nn[2] - ax[2] * nn[1], ax[2] * nn[0] - ax[0] * nn[2], ax[0] * nn[1] - ax[1] * nn[0]};
            const double l = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
            for (int i = 0; i < 3; i++) e1[i] /= l;
            const double e2[3] = {nn[1] * e1[2] - nn[2] * e1[1], nn[2] * e1[0] - nn[0] * e1[2], nn[0] * e1[1] - nn[1] * e1[0]};
            for (int i = 0; i < n_r; i++)
                for (int j = 0; j < n_t; j++) {
                    const double th = 2.0 * M_PI * (j + 0.5) / n_t, rr = a * gx[i];
                    const double w = gw[i] * gx[i] * (2.0 * M_PI / n_t) * a * a;
                    double4& d = disc[m * nq + i * n_t + j];
                    d.x = c[0] + rr * (std::cos(th) * e1[0] + std::sin(th) * e2[0]);
                    d.y = c[1] + rr * (std::cos(th) * e1[1] + std::sin(th) * e2[1]);
                    d.z = c[2] + rr * (std::cos(th) * e1[2] + std::sin(th) * e2[2]);
                    d.w = w;
                }
        }
        // double-float copies: disc points (hi, lo) and weights (re hi, re lo, im hi, im lo)
        auto split = [](double v, float& h, float& l) {
            h = (float)v;
            l = (float)(v - (double)h);
        };
        std::vector<float4> dsplit(2 * disc.size());
        for (size_t i = 0; i < disc.size(); i++) {
            float4& h = dsplit[i];
            float4& l = dsplit[disc.size() + i];
            split(disc[i].x, h.x, l.x);
            split(disc[i].y, h.y, l.y);
            split(disc[i].z, h.z, l.z);
            split(disc[i].w, h.w, l.w);
        }
        std::vector<float4> wsplit(ctx->tr_w.size() / 2);
        for (size_t i = 0; i < wsplit.size(); i++) {
            split(ctx->tr_w[2 * i], wsplit[i].x, wsplit[i].y);
            split(ctx->tr_w[2 * i + 1], wsplit[i].z, wsplit[i].w);
        }
        if ((rc = ctx->ensure_fardf()) || (rc = ctx->check_df_phase(ctx->k0re, true))) return rc;
        if (r0 == 0) {
            for (void* p : {(void*)S->disc, (void*)S->disc_df}) ctx->dfree(p);
            S->disc = (double4*)ctx->dalloc(disc.size() * sizeof(double4), &rc); if (rc) return rc;
            S->disc_df = (float4*)ctx->dalloc(dsplit.size() * sizeof(float4), &rc); if (rc) return rc;
            CK(cudaMemcpyAsync(S->disc, disc.data(), disc.size() * sizeof(double4), cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaMemcpyAsync(S->disc_df, dsplit.data(), dsplit.size() * sizeof(float4), cudaMemcpyHostToDevice,
                               ctx->stream));
        }
        // the weights of every excitation so far (joined ones included)
        for (void* p : {(void*)S->wdev, (void*)S->w_df}) ctx->dfree(p);
        S->wdev = (double2*)ctx->dalloc(ctx->tr_w.size() * sizeof(double), &rc); if (rc) return rc;
        S->w_df = (float4*)ctx->dalloc(std::max<size_t>(1, wsplit.size()) * sizeof(float4), &rc); if (rc) return rc;
        CK(cudaMemcpyAsync(S->wdev, ctx->tr_w.data(), ctx->tr_w.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(S->w_df, wsplit.data(), wsplit.size() * sizeof(float4), cudaMemcpyHostToDevice, ctx->stream));
        PistonArgs a{};
        a.pg = ctx->dev.pg64; a.tc = ctx->dev.tc; a.slot_v = ctx->dev.slot_v; a.slot_n = ctx->dev.slot_n;
        a.disc_h = S->disc_df; a.disc_l = S->disc_df + ne * nq; a.n_elem = (int)ne; a.nq = nq;
        a.w = S->w_df + r0 * ne;
        a.n_rhs = (int)count;
        {
            float h, l, hi, li;
            split(ctx->k0re, h, l);
            split(ctx->k0im, hi, li);
            a.k0 = make_float4(h, l, hi, li);
        }
        a.c = ctx->dfg.c; a.sctab = ctx->dfg.sctab; a.extab = ctx->dfg.extab;
        a.pref = make_double2(0.0, -ctx->omega_rho0 / (2.0 * M_PI));
        a.n_slots = g.n_slots;
        for (int q = 0; q < QP; q++)
            for (int k = 0; k < 3; k++) a.lam[q][k] = ctx->quad.lam[q][k];
        a.tri_out = S->tri_rhs;
        CK(cudaMemsetAsync(S->tri_rhs, 0, count * g.n_slots * 6 * sizeof(double2), ctx->stream));
        const dim3 grid((unsigned)((g.n_slots + PK_SLOTS - 1) / PK_SLOTS), (unsigned)((count + PK_RC - 1) / PK_RC));
        if (ctx->k0im != 0.0) piston_kernel<true><<<grid, PK_SLOTS * QP, 0, ctx->stream>>>(a);
        else piston_kernel<false><<<grid, PK_SLOTS * QP, 0, ctx->stream>>>(a);
        ctx->launches++;
    } else {
        return ctx->fail(BEM_ERR_STATE, "no incident field set");
    }
    CK(cudaGetLastError());
    for (int64_t r = 0; r < count; r++) {
        ReduceArgs ra{};
        ra.vc_ptr = ctx->dev.vc_ptr; ra.vc_idx = ctx->dev.vc_idx; ra.v_dof1 = ctx->dev.v_dof1;
        ra.v_dof2 = ctx->dev.v_dof2; ra.tri_out = S->tri_rhs + r * g.n_slots * 6; ra.v_begin = 0;
        ra.v_end = g.n_vert; ra.y = S->b + (r0 + r) * N;
        CK(launch_reduce(ra, ctx->stream));
        ctx->launches++;
    }
    ctx->rhs_ready = true;
    return BEM_OK;
}

void destroy_osrc_state(bem_ctx* ctx);
void set_osrc_tolerance(bem_ctx* ctx, double tol);

// Traces and incident-field data of excitation `rhs` of the last solve, for
// the field evaluation (k_field.cu).
int solve_field_inputs(bem_ctx* ctx, int64_t rhs, const double2** u, const double4** disc, const double2** wts,
                       int* n_elem, int* nq) {
    SolveState* S = ctx->solve;
    if (!S || S->n_rhs_solved == 0) return ctx->fail(BEM_ERR_STATE, "no solve has run");
    if (rhs < 0 || rhs >= S->n_rhs_solved) return ctx->fail(BEM_ERR_INVALID_ARG, "excitation index out of range");
    *u = S->u + rhs * ctx->geo.n_dof;
    *disc = S->disc;
    *n_elem = ctx->field_kind == 2 ? (int)ctx->tr_r.size() : 0;
    *nq = ctx->field_kind == 2 ? 32 : 0;
    *wts = ctx->field_kind == 2 ? S->wdev + rhs * (int64_t)ctx->tr_r.size() : nullptr;
    return BEM_OK;
}

namespace gbem {
// Solutions rhs0 .. rhs0+n-1 of the last solve into host memory (system order).
int copy_solution(bem_ctx* ctx, int64_t rhs0, int64_t n, double2* host) {
    SolveState* S = ctx->solve;
    if (!S || rhs0 < 0 || rhs0 + n > S->n_rhs_solved) return ctx->fail(BEM_ERR_STATE, "no such solution");
    const int64_t N = ctx->geo.n_dof;
    CK(cudaMemcpyAsync(host, S->u + rhs0 * N, n * N * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return BEM_OK;
}
}  // namespace gbem

namespace gbem {
// A superposition basis belongs to one transducer, mesh and set of materials.
void invalidate_basis(bem_ctx* ctx) {
    if (ctx->solve) ctx->solve->n_basis = 0;
}
// The operator changed: earlier (b, u) pairs no longer solve it.
void invalidate_recycle(bem_ctx* ctx) {
    if (ctx->solve) ctx->solve->rec_k = 0;
}
}  // namespace gbem

// Drop the solver objects after their device memory was released with the
// rest of the context's allocations.
void destroy_solver_state(bem_ctx* ctx) {
    delete ctx->solve;
    ctx->solve = nullptr;
    destroy_osrc_state(ctx);
}

static int ensure_solve_state(bem_ctx* ctx) {
    if (!ctx->solve) ctx->solve = new SolveState();
    SolveState* S = ctx->solve;
    const int64_t N = ctx->geo.n_dof;
    int rc;
    if (!S->r) {
        S->r = (double2*)ctx->dalloc(N * sizeof(double2), &rc); if (rc) return rc;
        S->d = (double2*)ctx->dalloc(N * sizeof(double2), &rc); if (rc) return rc;
        S->pb = (double2*)ctx->dalloc(N * sizeof(double2), &rc); if (rc) return rc;
    }
    return BEM_OK;
}


extern "C" {

int bem_set_plane_wave(bem_ctx* ctx, const double dir[3], bem_z amp) {
    if (!ctx || !dir) return BEM_ERR_INVALID_ARG;
    double n = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    if (!(n > 0)) return ctx->fail(BEM_ERR_INVALID_ARG, "zero plane-wave direction");
    for (int i = 0; i < 3; i++) ctx->pw_dir[i] = dir[i] / n;
    ctx->pw_amp[0] = amp.re;
    ctx->pw_amp[1] = amp.im;
    ctx->field_kind = 1;
    ctx->n_rhs = 1;
    ctx->rhs_ready = false;
    return BEM_OK;
}

int bem_set_transducer(bem_ctx* ctx, const double* c, const double* n, const double* r, int64_t n_elem,
                       double omega_rho0) {
    if (!ctx || !c || !n || !r || n_elem < 1) return BEM_ERR_INVALID_ARG;
    invalidate_basis(ctx);
    ctx->tr_c.assign(c, c + 3 * n_elem);
    ctx->tr_n.assign(n, n + 3 * n_elem);
    ctx->tr_r.assign(r, r + n_elem);
    ctx->omega_rho0 = omega_rho0;
    ctx->field_kind = 2;
    ctx->tr_w.assign(2 * n_elem, 0.0);
    for (int64_t m = 0; m < n_elem; m++) ctx->tr_w[2 * m] = 1.0;
    ctx->n_rhs = 1;
    ctx->rhs_ready = false;
    return BEM_OK;
}

int bem_set_excitations(bem_ctx* ctx, const bem_z* w, int64_t n_rhs) {
    if (!ctx || !w || n_rhs < 1) return BEM_ERR_INVALID_ARG;
    if (ctx->field_kind != 2) return ctx->fail(BEM_ERR_STATE, "set a transducer first");
    const int64_t ne = (int64_t)ctx->tr_r.size();
    ctx->tr_w.assign((const double*)w, (const double*)w + 2 * ne * n_rhs);
    ctx->n_rhs = n_rhs;
    ctx->rhs_ready = false;
    return BEM_OK;
}

int bem_rhs(bem_ctx* ctx, bem_z* b, int on_device) {
    if (!ctx || !b) return BEM_ERR_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    int rc = ctx->finalize();
    if (rc) return rc;
    if ((rc = ensure_solve_state(ctx))) return rc;
    if ((rc = build_rhs(ctx))) return rc;
    const int64_t n = (ctx->field_kind == 2 ? ctx->n_rhs : 1) * ctx->geo.n_dof;
    CK(cudaMemcpyAsync(b, ctx->solve->b, n * sizeof(double2), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       ctx->stream));
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
    return BEM_OK;
}

int bem_default_solve_opts(bem_solve_opts* o) {
    if (!o) return BEM_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof *o);
    o->restart = 100;
    o->max_iter = 2000;
    o->tol = 1e-8;
    o->precision = BEM_PREC_FP64;
    o->precondition = 1;
    o->inner_tol = 1e-4;
    o->max_refine = 10;
    o->operator_mode = 0;
    o->batch_rhs = 0;
    o->flexible = 1;
    o->prec_tol = 0.0;
    o->block_gmres = 0;
    return BEM_OK;
}

// Relative tolerance of one inner (FP32-operator) solve of the refinement
// when the FP64 residual is at rel: inner_tol, or looser once a smaller
// reduction already reaches the target (half of tol / rel), at most 1/2.
static double inner_tolerance(const bem_solve_opts& o, double rel) {
    const double need = rel > 0 ? 0.5 * o.tol / rel : o.inner_tol;
    return std::min(0.5, std::max(o.inner_tol, need));
}

// Work blocks for batched solves of up to R right-hand sides.
static int ensure_batch_state(bem_ctx* ctx, int64_t R) {
    SolveState* S = ctx->solve;
    if (S->batch_alloc >= R) return BEM_OK;
    for (void* p : {(void*)S->bt, (void*)S->bpb, (void*)S->bd, (void*)S->br}) ctx->dfree(p);
    S->bt = S->bpb = S->bd = S->br = nullptr;
    S->batch_alloc = 0;
    const size_t bytes = (size_t)R * ctx->geo.n_dof * sizeof(double2);
    int rc;
    S->bt = (double2*)ctx->dalloc(bytes, &rc); if (rc) return rc;
    S->bpb = (double2*)ctx->dalloc(bytes, &rc); if (rc) return rc;
    S->bd = (double2*)ctx->dalloc(bytes, &rc); if (rc) return rc;
    S->br = (double2*)ctx->dalloc(bytes, &rc); if (rc) return rc;
    S->batch_alloc = R;
    return BEM_OK;
}

// Solve R = nb right-hand sides b[R][N] into u[R][N] with R GMRES runs in
// lockstep (same method, tolerances and stopping rule per column as the
// one-at-a-time path).
// ---- recycled solution space (bem_solve_opts.recycle)

// Storage for `cap` pairs; a different capacity starts an empty space.
static int rec_ensure(bem_ctx* ctx, int64_t cap) {
    SolveState* S = ctx->solve;
    if (S->rec_cap == cap) return BEM_OK;
    for (void* p : {(void*)S->rec_Q, (void*)S->rec_U, (void*)S->rec_C}) ctx->dfree(p);
    S->rec_Q = S->rec_U = S->rec_C = nullptr;
    S->rec_cap = S->rec_k = 0;
    const int64_t N = ctx->geo.n_dof;
    int rc;
    S->rec_Q = (double2*)ctx->dalloc((size_t)cap * N * sizeof(double2), &rc); if (rc) return rc;
    S->rec_U = (double2*)ctx->dalloc((size_t)cap * N * sizeof(double2), &rc); if (rc) return rc;
    S->rec_C = (double2*)ctx->dalloc((size_t)cap * REC_RMAX * sizeof(double2), &rc); if (rc) return rc;
    S->rec_cap = cap;
    return BEM_OK;
}

// u_r = U' (Q^H b_r) for the R columns (the projection of b onto the earlier
// right-hand sides, solved by the same combination of their solutions); with
// res, also res_r = b_r - Q (Q^H b_r), its residual (A U' = Q to the earlier
// solves' tolerance, which the refinement's FP64 residuals then correct).
static int rec_start(bem_ctx* ctx, const double2* b, double2* u, int64_t R, double2* res) {
    SolveState* S = ctx->solve;
    const int64_t N = ctx->geo.n_dof;
    const int K = (int)S->rec_k;
    for (int64_t r0 = 0; r0 < R; r0 += REC_RMAX) {
        const int Rc = (int)std::min<int64_t>(REC_RMAX, R - r0);
        const dim3 grid((unsigned)((N + 255) / 256), (unsigned)Rc);
        rec_dots_kernel<<<dim3((unsigned)K, (unsigned)Rc), 256, 0, ctx->stream>>>(S->rec_Q, b + r0 * N, N, S->rec_C);
        rec_combine_kernel<<<grid, 256, 0, ctx->stream>>>(S->rec_U, K, S->rec_C, N, 1.0, nullptr, u + r0 * N);
        if (res) rec_combine_kernel<<<grid, 256, 0, ctx->stream>>>(S->rec_Q, K, S->rec_C, N, -1.0, b + r0 * N,
                                                                   res + r0 * N);
        ctx->launches += res ? 3 : 2;
    }
    CK(cudaGetLastError());
    return BEM_OK;
}

// Fold the solved pairs (b_r, u_r) into the space while it has room: two
// Gram-Schmidt passes of b_r against Q, the same combination applied to u_r,
// then both scaled by 1 / |b_r'| (A U' = Q holds to the solve tolerance).  A
// column within 1e-8 of the span adds nothing.  wb, wu: N-vector scratch.
static int rec_append(bem_ctx* ctx, const double2* b, const double2* u, int64_t R, double2* wb, double2* wu) {
    SolveState* S = ctx->solve;
    const int64_t N = ctx->geo.n_dof;
    const unsigned nb = (unsigned)((N + 255) / 256);
    for (int64_t r = 0; r < R && S->rec_k < S->rec_cap; r++) {
        double bn = 0;
        int rc = S->kry.norms(ctx, b + r * N, 1, &bn);
        if (rc) return rc;
        if (!(bn > 0)) continue;
        CK(cudaMemcpyAsync(wb, b + r * N, N * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(wu, u + r * N, N * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
        const int K = (int)S->rec_k;
        for (int pass = 0; pass < 2 && K > 0; pass++) {
            rec_dots_kernel<<<dim3((unsigned)K, 1), 256, 0, ctx->stream>>>(S->rec_Q, wb, N, S->rec_C);
            rec_combine_kernel<<<dim3(nb, 1), 256, 0, ctx->stream>>>(S->rec_Q, K, S->rec_C, N, -1.0, wb, wb);
            rec_combine_kernel<<<dim3(nb, 1), 256, 0, ctx->stream>>>(S->rec_U, K, S->rec_C, N, -1.0, wu, wu);
            ctx->launches += 3;
        }
        double wn = 0;
        if ((rc = S->kry.norms(ctx, wb, 1, &wn))) return rc;
        if (!(wn > 1e-8 * bn)) continue;
        rec_scale_kernel<<<nb, 256, 0, ctx->stream>>>(wb, N, 1.0 / wn, S->rec_Q + (int64_t)K * N);
        rec_scale_kernel<<<nb, 256, 0, ctx->stream>>>(wu, N, 1.0 / wn, S->rec_U + (int64_t)K * N);
        ctx->launches += 2;
        CK(cudaGetLastError());
        S->rec_k++;
    }
    return BEM_OK;
}

// cap > R (a single-batch mixed solve with ctx->join_hook set): before each
// refinement cycle the hook may hand over further excitations, which join as
// new columns (their right-hand sides built into b, zero start) until the
// block holds cap columns; R is then the final column count.
static int solve_block(bem_ctx* ctx, const bem_solve_opts& o, const double2* b, double2* u, int64_t& R,
                       bem_solve_report* rep, bool* converged, int64_t cap = 0) {
    SolveState* S = ctx->solve;
    const int64_t N = ctx->geo.n_dof;
    cap = std::max(cap, R);
    int rc;
    if ((rc = ensure_batch_state(ctx, cap))) return rc;
    if ((rc = S->kry.ensure(ctx, N, o.restart, cap))) return rc;
    auto plain = [ctx, &o, N](const double2* X, double2* Y, int prec, int64_t nr) -> int {
        if (o.operator_mode == 1)
            return prec == BEM_PREC_FP64 ? ctx->apply_assembled64(X, Y, nr) : ctx->apply_assembled(X, Y, nr);
        if (nr > 1) return prec == BEM_PREC_FP32 ? ctx->apply_ahat_multi(X, Y, nr) : ctx->apply_ahat64_multi(X, Y, nr);
        for (int64_t r = 0; r < nr; r++) {
            int e = ctx->apply_ahat(X + r * N, Y + r * N, prec);
            if (e) return e;
        }
        return BEM_OK;
    };
    const bool left = o.precondition && !o.flexible;
    auto op_for = [ctx, left, plain, S, &R](int prec) {
        return [ctx, prec, left, plain, S, &R](const double2* X, double2* Y) -> int {
            if (!left) return plain(X, Y, prec, R);
            int e = plain(X, S->bt, prec, R);
            return e ? e : ctx->apply_prec_batch(S->bt, Y, R);
        };
    };
    const Krylov::Op right = [ctx, &R](const double2* X, double2* Y) -> int { return ctx->apply_prec_batch(X, Y, R); };
    const Krylov::Op* rp = (o.precondition && o.flexible) ? &right : nullptr;
    auto rhs_of = [&](const double2* v) -> const double2* {
        if (!left) return v;
        rc = ctx->apply_prec_batch(v, S->bpb, R);
        return S->bpb;
    };
    auto residual = [&](std::vector<double>& rel, const std::vector<double>& bn) -> int {
        // br = b - A_hat u in FP64, relative column norms
        int e = plain(u, S->br, BEM_PREC_FP64, R);
        if (e) return e;
        if ((e = S->kry.axpby(ctx, 1.0, b, -1.0, S->br, S->br, R * N))) return e;
        std::vector<double> rn(R);
        if ((e = S->kry.norms(ctx, S->br, R, rn.data()))) return e;
        for (int64_t r = 0; r < R; r++) rel[r] = bn[r] > 0 ? rn[r] / bn[r] : 0.0;
        return BEM_OK;
    };
    std::vector<double> bn(cap), rel(cap, 1.0), irel(cap);
    std::vector<int> its(cap);
    if ((rc = S->kry.norms(ctx, b, R, bn.data()))) return rc;
    CK(cudaMemsetAsync(u, 0, R * N * sizeof(double2), ctx->stream));
    // recycled start: u = U' Q^H b, the part of b in the span of earlier right-hand sides
    if (o.recycle > 0 && (rc = rec_ensure(ctx, o.recycle))) return rc;
    const bool warm = o.recycle > 0 && S->rec_k > 0;
    if (warm && (rc = rec_start(ctx, b, u, R, o.precision == BEM_PREC_FP64 ? nullptr : S->br))) return rc;
    int it = 0;
    double worst = 0;
    // block GMRES, or R GMRES runs in lockstep (also where the block's
    // starting residuals are dependent columns)
    auto inner_solve = [&](const Krylov::Op& op, const double2* rhs, double2* x, double tol_in, bool zero_guess,
                           bool fp32_basis) -> int {
        if (o.block_gmres) {
            bool deficient = false;
            const int e = S->kry.gmres_block(ctx, op, rhs, x, R, o.restart, tol_in, o.max_iter - it, its.data(),
                                             irel.data(), zero_guess, rp, fp32_basis, &deficient);
            if (e || !deficient) return e;
        }
        return S->kry.gmres_batch(ctx, op, rhs, x, R, o.restart, tol_in, o.max_iter - it, its.data(), irel.data(),
                                  zero_guess, rp);
    };
    if (o.precision == BEM_PREC_FP64) {
        const double2* sb = rhs_of(b);
        if (rc) return rc;
        double inner = o.tol;
        for (int attempt = 0; attempt < 4; attempt++) {
            if ((rc = inner_solve(op_for(BEM_PREC_FP64), sb, u, inner, attempt == 0 && !warm, false))) return rc;
            it += *std::max_element(its.begin(), its.begin() + R);
            for (int64_t r = 0; r < R; r++) rep->iterations += its[r];
            if ((rc = residual(rel, bn))) return rc;
            worst = *std::max_element(rel.begin(), rel.begin() + R);
            if (worst <= o.tol || it >= o.max_iter) break;
            inner *= 0.1;
        }
    } else {
        if (warm) {  // br = b - Q Q^H b from rec_start
            std::vector<double> rn(R);
            if ((rc = S->kry.norms(ctx, S->br, R, rn.data()))) return rc;
            for (int64_t r = 0; r < R; r++) rel[r] = bn[r] > 0 ? rn[r] / bn[r] : 0.0;
        } else {
            CK(cudaMemcpyAsync(S->br, b, R * N * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
            for (int64_t r = 0; r < R; r++) rel[r] = bn[r] > 0 ? 1.0 : 0.0;
        }
        int ref = 0, inner_prec = BEM_PREC_FP32;
        double prev = 2.0;
        for (; ref <= o.max_refine; ref++) {
            if (R < cap && ctx->join_hook) {
                // excitations that arrived while this block ran join it here
                std::vector<double> w;
                const int64_t k = ctx->join_hook(cap - R, w);
                if (k > 0) {
                    ctx->tr_w.insert(ctx->tr_w.end(), w.begin(), w.end());
                    ctx->n_rhs += k;
                    if ((rc = build_rhs(ctx, R, k))) return rc;
                    if ((rc = S->kry.norms(ctx, b + R * N, k, bn.data() + R))) return rc;
                    CK(cudaMemsetAsync(u + R * N, 0, k * N * sizeof(double2), ctx->stream));
                    CK(cudaMemcpyAsync(S->br + R * N, b + R * N, k * N * sizeof(double2), cudaMemcpyDeviceToDevice,
                                       ctx->stream));
                    for (int64_t r = R; r < R + k; r++) rel[r] = bn[r] > 0 ? 1.0 : 0.0;
                    R += k;
                    prev = 2.0;  // new columns start at residual 1: not a stalled refinement
                    ref = std::min(ref, std::max(0, o.max_refine - 2));  // and get refinement cycles of their own
                }
            }
            worst = *std::max_element(rel.begin(), rel.begin() + R);
            if (worst <= o.tol || it >= o.max_iter || ref == o.max_refine) break;
            // stalled refinement (reduced-precision operator error too large
            // for this conditioning): the remaining inner solves run in FP64
            if (worst > 0.5 * prev) inner_prec = BEM_PREC_FP64;
            prev = worst;
            const double2* sr = rhs_of(S->br);
            if (rc) return rc;
            if ((rc = inner_solve(op_for(inner_prec), sr, S->bd, inner_tolerance(o, worst), true,
                                  inner_prec != BEM_PREC_FP64)))
                return rc;
            it += *std::max_element(its.begin(), its.begin() + R);
            for (int64_t r = 0; r < R; r++) rep->iterations += its[r];
            if ((rc = S->kry.axpby(ctx, 1.0, u, 1.0, S->bd, u, R * N))) return rc;
            if ((rc = residual(rel, bn))) return rc;
        }
        rep->refinements += ref;
    }
    if (o.recycle > 0 && worst <= o.tol) {  // keep the solved pairs for later solves of this operator
        if ((rc = rec_ensure(ctx, o.recycle))) return rc;
        if ((rc = rec_append(ctx, b, u, R, S->bt, S->bpb))) return rc;
    }
    rep->residual = std::max(rep->residual, worst);
    *converged &= worst <= o.tol;
    return BEM_OK;
}

int bem_solve(bem_ctx* ctx, const bem_solve_opts* opts, bem_solve_report* rep) {
    if (!ctx) return BEM_ERR_INVALID_ARG;
    bem_solve_opts o;
    bem_default_solve_opts(&o);
    if (opts) o = *opts;
    if (o.restart < 1 || o.max_iter < 1 || !(o.tol > 0) || (o.precision != BEM_PREC_FP64 && o.precision != BEM_PREC_FP32) ||
        o.operator_mode < 0 || o.operator_mode > 2 || o.batch_rhs < 0 || o.flexible < 0 || o.flexible > 1 ||
        !(o.prec_tol >= 0) || o.prec_tol >= 1 || o.block_gmres < 0 || o.block_gmres > 1 || o.recycle < 0)
        return ctx->fail(BEM_ERR_INVALID_ARG, "bad solve options");
    CK(cudaSetDevice(ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    int rc = ctx->finalize();
    if (rc) return rc;
    if ((rc = ctx->ensure_near())) return rc;
    if ((rc = ensure_solve_state(ctx))) return rc;
    // a request loop may hand excitations to a running mixed solve (joined at
    // refinement boundaries) while it is a single batch: room for a full block
    const int64_t nr0 = ctx->field_kind == 2 ? ctx->n_rhs : 1;
    const int64_t join_cap = std::max<int64_t>(1, solve_batch_width(o, std::max<int64_t>(o.batch_rhs, 1)));
    const bool joinable = ctx->join_hook && o.precision == BEM_PREC_FP32 && ctx->field_kind == 2 && nr0 <= join_cap &&
                          o.batch_rhs > 1;
    if ((rc = build_rhs(ctx, 0, -1, joinable ? join_cap : 0))) return rc;
    SolveState* S = ctx->solve;
    const int64_t N = ctx->geo.n_dof, nr = nr0;
    o.operator_mode = resolved_operator_mode(o.operator_mode, N);
    if ((rc = S->kry.ensure(ctx, N, o.restart))) return rc;
    // the preconditioner only has to be a fixed linear map to the accuracy the
    // GMRES it sits in needs: two orders below that GMRES's tolerance
    // inside a flexible GMRES the preconditioner may be any map, so a sparse
    // solve that stops short (iteration cap, breakdown) keeps its iterate
    struct TolScope {
        bem_ctx* c;
        double saved;
        bool strict;
        ~TolScope() {
            set_osrc_tolerance(c, saved);
            c->osrc_strict = strict;
        }
    } tol_scope{ctx, ctx->osrc_tol, ctx->osrc_strict};
    ctx->osrc_strict = !(o.precondition && o.flexible);
    const double gm_tol = o.precision == BEM_PREC_FP64 ? o.tol : std::max(o.inner_tol, o.tol);
    set_osrc_tolerance(ctx, o.prec_tol > 0 ? o.prec_tol : o.flexible ? 0.3 : std::max(1e-13, 0.01 * gm_tol));
    bem_solve_report R{};
    bool converged = true;
    // the operator of one precision level: matrix-free or assembled, then the preconditioner
    auto plain = [ctx, &o](const double2* x, double2* y, int prec) -> int {
        if (o.operator_mode == 1)
            return prec == BEM_PREC_FP64 ? ctx->apply_assembled64(x, y, 1) : ctx->apply_assembled(x, y, 1);
        return ctx->apply_ahat(x, y, prec);
    };
    const bool left = o.precondition && !o.flexible;
    auto op_for = [ctx, left, plain](int prec) {
        return [ctx, prec, left, plain](const double2* x, double2* y) -> int {
            if (!left) return plain(x, y, prec);
            int r = plain(x, ctx->dev.ys2, prec);
            return r ? r : ctx->apply_prec(ctx->dev.ys2, y);
        };
    };
    const Krylov::Op right = [ctx](const double2* x, double2* y) -> int { return ctx->apply_prec(x, y); };
    const Krylov::Op* rp = (o.precondition && o.flexible) ? &right : nullptr;
    int64_t n_solved = nr;
    if (joinable) {
        int64_t Rb = nr;
        if ((rc = solve_block(ctx, o, S->b, S->u, Rb, &R, &converged, join_cap))) return rc;
        n_solved = Rb;
    } else if (o.batch_rhs > 1 && nr > 1) {
        // blocks of up to batch_rhs excitations, GMRES in lockstep; block GMRES
        // takes at most BLOCK_COLS columns per block (its host-side band QR
        // update costs O(step x P^3)), the batch split evenly
        const int64_t width = solve_batch_width(o, nr);
        for (int64_t r0 = 0; r0 < nr; r0 += width) {
            int64_t Rb = std::min<int64_t>(width, nr - r0);
            if ((rc = solve_block(ctx, o, S->b + r0 * N, S->u + r0 * N, Rb, &R, &converged))) return rc;
        }
    }
    for (int64_t r = 0; r < (joinable || (o.batch_rhs > 1 && nr > 1) ? 0 : nr); r++) {
        const double2* b = S->b + r * N;
        double2* u = S->u + r * N;
        double bnorm;
        if ((rc = S->kry.norm(ctx, b, &bnorm))) return rc;
        // right-hand side of the system GMRES sees
        auto rhs_of = [&](const double2* v) -> const double2* {
            if (!left) return v;
            rc = ctx->apply_prec(v, S->pb);
            return S->pb;
        };
        if (o.precision == BEM_PREC_FP64) {
            // plain FP64: GMRES on (P) A_hat u = (P) b until the true residual meets tol
            CK(cudaMemsetAsync(u, 0, N * sizeof(double2), ctx->stream));
            const double2* sb = rhs_of(b);
            if (rc) return rc;
            int it = 0;
            double rel = 1;
            double inner = o.tol;
            for (int attempt = 0; attempt < 4; attempt++) {
                int its = 0;
                if ((rc = S->kry.gmres(ctx, op_for(BEM_PREC_FP64), sb, u, o.restart, inner, o.max_iter - it, &its, &rel,
                                       attempt == 0, rp)))
                    return rc;
                it += its;
                // true FP64 residual of the unpreconditioned system
                if ((rc = plain(u, S->r, BEM_PREC_FP64))) return rc;
                if ((rc = S->kry.axpby(ctx, 1.0, b, -1.0, S->r, S->r))) return rc;
                double rn;
                if ((rc = S->kry.norm(ctx, S->r, &rn))) return rc;
                rel = rn / bnorm;
                if (rel <= o.tol || it >= o.max_iter) break;
                inner *= 0.1;
            }
            R.iterations += it;
            R.residual = std::max(R.residual, rel);
            converged &= rel <= o.tol;
        } else {
            // mixed: FP32 inner GMRES, FP64 residual refinement
            CK(cudaMemsetAsync(u, 0, N * sizeof(double2), ctx->stream));
            CK(cudaMemcpyAsync(S->r, b, N * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
            double rel = 1.0, prev = 2.0;
            int it = 0, ref = 0, inner_prec = BEM_PREC_FP32;
            for (; ref <= o.max_refine; ref++) {
                double rn;
                if ((rc = S->kry.norm(ctx, S->r, &rn))) return rc;
                rel = rn / bnorm;
                if (rel <= o.tol || it >= o.max_iter) break;
                if (ref == o.max_refine) break;
                // refinement stalls when the reduced-precision operator's error
                // times the conditioning is near 1: finish in FP64
                if (rel > 0.5 * prev) inner_prec = BEM_PREC_FP64;
                prev = rel;
                const double2* sr = rhs_of(S->r);
                if (rc) return rc;
                int its = 0;
                double irel = 0;
                if ((rc = S->kry.gmres(ctx, op_for(inner_prec), sr, S->d, o.restart, inner_tolerance(o, rel),
                                       o.max_iter - it, &its, &irel, true, rp)))
                    return rc;
                it += its;
                if ((rc = S->kry.axpby(ctx, 1.0, u, 1.0, S->d, u))) return rc;
                if ((rc = plain(u, S->r, BEM_PREC_FP64))) return rc;
                if ((rc = S->kry.axpby(ctx, 1.0, b, -1.0, S->r, S->r))) return rc;
            }
            R.iterations += it;
            R.refinements += ref;
            R.residual = std::max(R.residual, rel);
            converged &= rel <= o.tol;
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    if ((rc = ctx->check_device_error())) return rc;
    S->n_rhs_solved = n_solved;
    R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = R;
    if (!converged) return ctx->fail(BEM_ERR_NOT_CONVERGED, "GMRES did not reach the requested residual");
    return BEM_OK;
}

// ---- excitation superposition (treatment planning: many phase patterns of one array)
//
// The traces are linear in the piston weights (the right-hand side is a sum of
// the pistons' Rayleigh fields, eq. Galerkin_disc_rhs1, and A_hat does not
// depend on the excitation), so once the solution u_m of every piston m alone
// is known, any weight vector w gives u = sum_m w_m u_m: one complex GEMM
// instead of a solve.

int bem_solve_basis(bem_ctx* ctx, const bem_solve_opts* opts, bem_solve_report* rep) {
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (ctx->field_kind != 2) return ctx->fail(BEM_ERR_STATE, "set a transducer first");
    const int64_t ne = (int64_t)ctx->tr_r.size();
    // unit excitations, restoring the caller's weights afterwards
    const std::vector<double> saved_w = ctx->tr_w;
    const int64_t saved_n = ctx->n_rhs;
    std::vector<double> eye((size_t)2 * ne * ne, 0.0);
    for (int64_t m = 0; m < ne; m++) eye[(size_t)2 * (m * ne + m)] = 1.0;
    int rc = bem_set_excitations(ctx, (const bem_z*)eye.data(), ne);
    if (!rc) rc = bem_solve(ctx, opts, rep);
    const int solve_rc = rc;
    if (!rc || rc == BEM_ERR_NOT_CONVERGED) {
        SolveState* S = ctx->solve;
        const int64_t N = ctx->geo.n_dof;
        if (S->n_basis != ne) {
            ctx->dfree(S->basis);
            S->basis = (double2*)ctx->dalloc((size_t)ne * N * sizeof(double2), &rc);
            if (rc) {
                S->basis = nullptr;
                S->n_basis = 0;
            }
        }
        if (!rc && !ctx->df_exp) {
            ctx->df_exp = (int*)ctx->dalloc(2 * sizeof(int), &rc);
            if (rc) ctx->df_exp = nullptr;
        }
        if (!rc) {
            // kept in the split form of k_df64.cu for bem_superpose
            CK(cudaMemcpyAsync(S->basis, S->u, (size_t)ne * N * sizeof(double2), cudaMemcpyDeviceToDevice,
                               ctx->stream));
            rc = df_prepare_inplace(ctx, S->basis, ne * N, ctx->df_exp + 1);
            if (!rc) CK(cudaStreamSynchronize(ctx->stream));
            if (!rc) {
                S->n_basis = ne;
                rc = solve_rc;
            }
        }
    }
    ctx->tr_w = saved_w;
    ctx->n_rhs = saved_n;
    ctx->rhs_ready = false;
    return rc;
}

int bem_superpose(bem_ctx* ctx, const bem_z* w, int64_t n_exc, bem_z* u, int on_device) {
    if (!ctx || !w || !u || n_exc < 1) return BEM_ERR_INVALID_ARG;
    SolveState* S = ctx->solve;
    const int64_t ne = (int64_t)ctx->tr_r.size();
    if (!S || !S->basis || S->n_basis != ne || ctx->field_kind != 2)
        return ctx->fail(BEM_ERR_STATE, "no superposition basis: call bem_solve_basis after bem_set_transducer");
    CK(cudaSetDevice(ctx->device));
    const int64_t N = ctx->geo.n_dof;
    const double2* wd = (const double2*)w;
    double2* ud = (double2*)u;
    int rc;
    if (!on_device) {
        const size_t need = ((size_t)n_exc * ne + (size_t)n_exc * N) * sizeof(double2);
        if (need > S->wstage_bytes) {
            ctx->dfree(S->wstage);
            S->wstage = (double2*)ctx->dalloc(need, &rc);
            if (rc) {
                S->wstage = nullptr;
                S->wstage_bytes = 0;
                return rc;
            }
            S->wstage_bytes = need;
        }
        CK(cudaMemcpyAsync(S->wstage, w, (size_t)n_exc * ne * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
        wd = S->wstage;
        ud = S->wstage + n_exc * ne;
    }
    // U = W B with the basis in the split form of k_df64.cu (FP64 accuracy)
    if ((rc = df_combine(ctx, (const float4*)S->basis, ctx->df_exp + 1, ne, N, wd, n_exc, ud))) return rc;
    if (!on_device) {
        CK(cudaMemcpyAsync(u, ud, (size_t)n_exc * N * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return BEM_OK;
}

int bem_get_solution(bem_ctx* ctx, int64_t rhs, bem_z* u, int on_device) {
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!ctx->solve || ctx->solve->n_rhs_solved == 0) return ctx->fail(BEM_ERR_STATE, "no solve has run");
    if (rhs < 0 || rhs >= ctx->solve->n_rhs_solved || !u) return ctx->fail(BEM_ERR_INVALID_ARG, "bad solution request");
    const int64_t N = ctx->geo.n_dof;
    CK(cudaMemcpyAsync(u, ctx->solve->u + rhs * N, N * sizeof(double2),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return BEM_OK;
}

int bem_get_traces(bem_ctx* ctx, int32_t dom, int64_t rhs, bem_z* dirichlet, bem_z* neumann, int on_device) {
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!ctx->solve || ctx->solve->n_rhs_solved == 0) return ctx->fail(BEM_ERR_STATE, "no solve has run");
    if (dom < 0 || dom >= ctx->geo.n_dom || rhs < 0 || rhs >= ctx->solve->n_rhs_solved || !dirichlet || !neumann)
        return ctx->fail(BEM_ERR_INVALID_ARG, "bad trace request");
    const int64_t N = ctx->geo.n_dof, off = ctx->geo.dom_dof_off[dom], nv = ctx->geo.dom_nv[dom];
    const double2* u = ctx->solve->u + rhs * N;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(neumann, u + off, nv * sizeof(double2), k, ctx->stream));
    CK(cudaMemcpyAsync(dirichlet, u + off + nv, nv * sizeof(double2), k, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return BEM_OK;
}

}  // extern "C"
