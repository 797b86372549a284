// k_field.cu -- pressure at arbitrary points from the solved traces.
//
// Representation formula (paper App. A, eq. rep_formula_gen) with the
// PMCHWT jump potentials: outside every domain
//   p_tot(x) = p_inc(x) + DL_k0(gamma_D p_tot)(x) - SL_k0(gamma_N^+ p_tot)(x)
// over all surfaces, and inside domain j
//   p^j(x) = SL_kj((rho_j/rho_0) gamma_N^+ p_tot)(x) - DL_kj(gamma_D p_tot)(x)
// over the surface of domain j (interior traces by eq. Form1_BCs); SL, DL
// with G = exp(ikr)/(4 pi r).  Surface integrals use the regular rule with
// the trial densities of the operator application (gather kernel), in FP32
// with the tile-local phase of the far-field kernel; the regular rule loses
// accuracy for points within about one element size of a surface.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "ctx.h"
#include "internal.h"
#include "pair_math.h"

namespace gbem {

struct FieldArgs {
    const double* pts;      // [n][3]
    const int32_t* dom;     // [n] -1 exterior, else domain
    int64_t n;
    const float4* pg;       // source points (dx, dy, dz, w), pair-interleaved
    const float4* pd;       // densities (w psi, w phi), pair-interleaved
    const float4* tg;       // triangles (n, h)
    const double4* tc;
    const int* tntri;
    const int* tdom;
    const double2* kdom;
    const double* rho_ratio; // [n_dom]
    int n_dom;
    int* err;                // device error flag: value 4 or-ed in for a domain id out of range
    double2 k0;
    int n_tiles;
    int inc_kind;            // 1 plane wave, 2 pistons
    double pw_d[3];
    double2 pw_amp;
    const double4* disc;     // piston points (x, y, z, weight)
    const double2* wts;      // piston weights of this excitation
    int n_elem, nq;
    double2 pref;
    double2* out;
    int chunk_tiles;         // source tiles per grid.y index of the partial kernel
    int n_chunks;
    float4* partial;         // [n_chunks][n] (SL re, im, DL re, im) per source chunk
};

__device__ __forceinline__ float f_reduce_phase(double t) {
    const double two_pi_hi = 6.283185307179586, two_pi_lo = 2.4492935982947064e-16;
    double nn = rint(t * 0.15915494309189535);
    double r = fma(-nn, two_pi_hi, t);
    r = fma(-nn, two_pi_lo, r);
    return (float)r;
}

// One point against one source tile, two source points per packed FP32
// instruction: the single-layer sum over the tile and, per triangle, the
// double-layer sum n_t.(y - x) F sigma_D.  With D = x - c_source (2D in
// D2x..z), a source offset g from its tile centre gives
// r^2 - R_c^2 = g.(g - 2D).  As in the far-field kernel, -F is formed:
// -Re F = P Gr + B Gi, -Im F = P Gi - B Gr with P = Im k / r + 1/r^2,
// B = Re k / r.
template <bool LOSSY>
__device__ __forceinline__ void field_tile(const float4* s_pg, const float4* s_pd, const float4* s_tg, int ntri,
                                           float D2x, float D2y, float D2z, f2 Rc2, f2 Rc, f2 th, f2 kr, f2 nkr, f2 ki,
                                           f2 nkil2, float& slr, float& sli, float& dlr, float& dli) {
    const f2 m2x = bc2(-D2x), m2y = bc2(-D2y), m2z = bc2(-D2z);
    const f2 z2 = make_float2(0.f, 0.f);
    f2 Vr = z2, Vi = z2;
    for (int tl = 0; tl < ntri; tl++) {
        const float4 tgv = s_tg[tl];
        const float fK = tgv.w - 0.5f * (tgv.x * D2x + tgv.y * D2y + tgv.z * D2z);  // n_t.(y - x)
        f2 nS1r = z2, nS1i = z2;
#pragma unroll
        for (int j = 0; j < QP / 2; j++) {
            const float4 GA = s_pg[tl * QP + 2 * j], GB = s_pg[tl * QP + 2 * j + 1];
            const float4 DA = s_pd[tl * QP + 2 * j], DB = s_pd[tl * QP + 2 * j + 1];
            const f2 gx = lo2(GA), gy = hi2(GA), gz = lo2(GB);
            const f2 d1r = lo2(DA), d1i = hi2(DA), d2r = lo2(DB), d2i = hi2(DB);
            const f2 s = fma2(gx, add2(gx, m2x), fma2(gy, add2(gy, m2y), mul2(gz, add2(gz, m2z))));
            const f2 r2 = add2(s, Rc2);
            const f2 rinv = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
            const f2 den = fma2(r2, rinv, Rc);  // r + R_c
            const f2 rho = mul2(s, make_float2(rcp_approx(den.x), rcp_approx(den.y)));
            const f2 arg = fma2(kr, rho, th);
            f2 sn, cs;
            sincos_approx(arg.x, &sn.x, &cs.x);
            sincos_approx(arg.y, &sn.y, &cs.y);
            const f2 rinv2 = mul2(rinv, rinv);
            f2 am = rinv;
            if constexpr (LOSSY) {
                const f2 e = mul2(nkil2, mul2(r2, rinv));
                am = mul2(make_float2(ex2_approx(e.x), ex2_approx(e.y)), rinv);
            }
            const f2 Gr = mul2(am, cs), Gi = mul2(am, sn);
            const f2 nd1i = neg2(d1i), nd2i = neg2(d2i);
            Vr = fma2(Gr, d1r, fma2(Gi, nd1i, Vr));
            Vi = fma2(Gr, d1i, fma2(Gi, d1r, Vi));
            const f2 P = LOSSY ? fma2(ki, rinv, rinv2) : rinv2;
            const f2 B = mul2(kr, rinv), nB = mul2(nkr, rinv);
            const f2 nFr = fma2(P, Gr, mul2(B, Gi)), nFi = fma2(P, Gi, mul2(nB, Gr));
            nS1r = fma2(nFr, d2r, fma2(nFi, nd2i, nS1r));
            nS1i = fma2(nFr, d2i, fma2(nFi, d2r, nS1i));
        }
        dlr = fmaf(-fK, nS1r.x + nS1r.y, dlr);
        dli = fmaf(-fK, nS1i.x + nS1i.y, dli);
    }
    slr += Vr.x + Vr.y;
    sli += Vi.x + Vi.y;
}

// Pass 1: the surface potentials of one block of TP points from one chunk of
// source tiles (grid: point blocks x source chunks, so that a small set of
// points still fills the GPU).
__global__ void __launch_bounds__(TP) field_partial_kernel(FieldArgs a) {
    __shared__ float4 s_pg[TP], s_pd[TP], s_tg[TT];
    const int64_t i = (int64_t)blockIdx.x * TP + threadIdx.x;
    const bool live = i < a.n;
    double x = 0, y = 0, z = 0;
    int dom = -1;
    if (live) {
        x = a.pts[3 * i];
        y = a.pts[3 * i + 1];
        z = a.pts[3 * i + 2];
        dom = a.dom[i];
    }
    const bool bad = live && (dom < -1 || dom >= a.n_dom);  // device-side ids are checked here
    const bool use = live && !bad;
    if (bad) dom = -1;
    const double2 k = dom < 0 ? a.k0 : a.kdom[dom];
    const bool lossy = k.y != 0.0;
    const f2 kr2 = bc2((float)k.x), nkr2 = bc2((float)-k.x), ki2 = bc2((float)k.y);
    const f2 nkil2 = bc2((float)(-k.y * 1.4426950408889634));
    float slr = 0, sli = 0, dlr = 0, dli = 0;
    const int s_begin = blockIdx.y * a.chunk_tiles, s_end = min(s_begin + a.chunk_tiles, a.n_tiles);
    for (int s = s_begin; s < s_end; s++) {
        __syncthreads();
        const int64_t pb = (int64_t)s * TP;
        s_pg[threadIdx.x] = a.pg[pb + threadIdx.x];
        s_pd[threadIdx.x] = a.pd[pb + threadIdx.x];
        if (threadIdx.x < TT) s_tg[threadIdx.x] = a.tg[(int64_t)s * TT + threadIdx.x];
        __syncthreads();
        if (!use || (dom >= 0 && a.tdom[s] != dom)) continue;
        const double4 c = a.tc[s];
        const double Dx = x - c.x, Dy = y - c.y, Dz = z - c.z;  // x - c_source
        const double R = sqrt(Dx * Dx + Dy * Dy + Dz * Dz);
        const float D2x = (float)(2 * Dx), D2y = (float)(2 * Dy), D2z = (float)(2 * Dz);
        const float Rc2 = (float)(R * R), Rc = (float)R, th = f_reduce_phase(k.x * R);
        const int ntri = a.tntri[s];
        if (lossy)
            field_tile<true>(s_pg, s_pd, s_tg, ntri, D2x, D2y, D2z, bc2(Rc2), bc2(Rc), bc2(th), kr2, nkr2, ki2, nkil2,
                             slr, sli, dlr, dli);
        else
            field_tile<false>(s_pg, s_pd, s_tg, ntri, D2x, D2y, D2z, bc2(Rc2), bc2(Rc), bc2(th), kr2, nkr2, ki2, nkil2,
                              slr, sli, dlr, dli);
    }
    if (live) a.partial[(int64_t)blockIdx.y * a.n + i] = make_float4(slr, sli, dlr, dli);
    if (bad && blockIdx.y == 0) atomicOr(a.err, 4);
}

// Pass 2, one thread per point: the chunks summed in chunk order (compensated
// FP32 sums, converted to FP64 once), the representation formula's
// combination and the incident field.
__global__ void field_finish_kernel(FieldArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double x = a.pts[3 * i], y = a.pts[3 * i + 1], z = a.pts[3 * i + 2];
    const int dom = a.dom[i];
    if (dom < -1 || dom >= a.n_dom) {  // reported through the error flag by the partial kernel
        a.out[i] = make_double2(__longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll));
        return;
    }
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    for (int ch = 0; ch < a.n_chunks; ch++) {
        const float4 v = a.partial[(int64_t)ch * a.n + i];
        const float xv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const float u = hi[c] + xv[c];  // TwoSum: hi + x = u + (rounding error)
            const float xb = u - hi[c];
            lo[c] += (hi[c] - (u - xb)) + (xv[c] - xb);
            hi[c] = u;
        }
    }
    const double slr = (double)hi[0] + lo[0], sli = (double)hi[1] + lo[1];
    const double dlr = (double)hi[2] + lo[2], dli = (double)hi[3] + lo[3];
    const double inv4pi = 0.07957747154594767;
    double pr, pi;
    if (dom >= 0) {
        const double rr = a.rho_ratio[dom];
        pr = inv4pi * (rr * slr - dlr);
        pi = inv4pi * (rr * sli - dli);
    } else {
        pr = inv4pi * (dlr - slr);
        pi = inv4pi * (dli - sli);
        if (a.inc_kind == 1) {
            const double ph = a.pw_d[0] * x + a.pw_d[1] * y + a.pw_d[2] * z;
            double sn, cs;
            sincos(a.k0.x * ph, &sn, &cs);
            const double m = exp(-a.k0.y * ph);
            pr += m * (a.pw_amp.x * cs - a.pw_amp.y * sn);
            pi += m * (a.pw_amp.x * sn + a.pw_amp.y * cs);
        } else if (a.inc_kind == 2) {
            double qr = 0, qi = 0;
            for (int e = 0; e < a.n_elem; e++) {
                double er = 0, ei = 0;
                for (int j = 0; j < a.nq; j++) {
                    const double4 d = a.disc[(int64_t)e * a.nq + j];
                    const double ex = x - d.x, ey = y - d.y, ez = z - d.z;
                    const double R = sqrt(ex * ex + ey * ey + ez * ez);
                    double sn, cs;
                    sincos(a.k0.x * R, &sn, &cs);
                    const double amp = exp(-a.k0.y * R) / R * d.w;
                    er += amp * cs;
                    ei += amp * sn;
                }
                const double2 w = a.wts[e];
                qr += w.x * er - w.y * ei;
                qi += w.x * ei + w.y * er;
            }
            pr += a.pref.x * qr - a.pref.y * qi;
            pi += a.pref.x * qi + a.pref.y * qr;
        }
    }
    a.out[i] = make_double2(pr, pi);
}

// Source chunks per launch: enough CTAs for about eight per SM over the GPU
// (152 SMs on GB300, read from the device), each chunk at least one tile.
int field_chunks(int64_t n_points, int n_tiles, int n_sm) {
    const int64_t blocks = (n_points + TP - 1) / TP;
    int64_t want = (8LL * n_sm + blocks - 1) / blocks;
    if (want < 1) want = 1;
    if (want > n_tiles) want = n_tiles;
    return (int)want;
}

cudaError_t launch_field(const FieldArgs& a, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    field_partial_kernel<<<dim3((unsigned)((a.n + TP - 1) / TP), (unsigned)a.n_chunks), TP, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    field_finish_kernel<<<(unsigned)((a.n + 127) / 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gbem

using namespace gbem;

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int solve_field_inputs(bem_ctx* ctx, int64_t rhs, const double2** u, const double4** disc, const double2** wts,
                       int* n_elem, int* nq);

extern "C" int bem_field(bem_ctx* ctx, int64_t rhs, const double* points, const int32_t* domain_of_point,
                         int64_t n_points, bem_z* out, int on_device) {
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (n_points < 0 || (n_points > 0 && (!points || !domain_of_point || !out)))
        return ctx->fail(BEM_ERR_INVALID_ARG, "bad field arguments");
    if (n_points == 0) return BEM_OK;
    CK(cudaSetDevice(ctx->device));
    const double2* u = nullptr;
    const double4* disc = nullptr;
    const double2* wts = nullptr;
    int n_elem = 0, nq = 0;
    int rc = solve_field_inputs(ctx, rhs, &u, &disc, &wts, &n_elem, &nq);
    if (rc) return rc;
    const Geometry& g = ctx->geo;
    // check the domain ids of a host array here; the kernels check device arrays
    if (!on_device)
        for (int64_t i = 0; i < n_points; i++)
            if (domain_of_point[i] < -1 || domain_of_point[i] >= g.n_dom)
                return ctx->fail(BEM_ERR_INVALID_ARG, "domain id of a point out of range");
    // trial densities of the traces
    GatherArgs ga{};
    ga.slot_v = ctx->dev.slot_v; ga.v_dof1 = ctx->dev.v_dof1; ga.v_dof2 = ctx->dev.v_dof2; ga.pt_w = ctx->dev.pt_w;
    ga.slot_curl = ctx->dev.slot_curl; ga.x = u; ga.s_begin = 0; ga.s_end = g.n_slots;
    for (int q = 0; q < QP; q++)
        for (int kk = 0; kk < 3; kk++) ga.lam[q][kk] = ctx->quad.lam[q][kk];
    ga.pd32 = ctx->dev.pd32; ga.tcurl32 = ctx->dev.tcurl32;
    CK(launch_gather(ga, ctx->stream));
    // one grow-only scratch buffer: chunk partials | output | points | rho ratios | domain ids
    int n_sm = 0;
    CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->device));
    const int want = field_chunks(n_points, g.n_tiles, n_sm);
    const int chunk_tiles = (g.n_tiles + want - 1) / want;
    const int n_chunks = (g.n_tiles + chunk_tiles - 1) / chunk_tiles;
    auto up16 = [](size_t b) { return (b + 15) / 16 * 16; };
    const size_t b_part = up16((size_t)n_chunks * n_points * sizeof(float4));
    const size_t b_out = on_device ? 0 : up16((size_t)n_points * sizeof(double2));
    const size_t b_pts = on_device ? 0 : up16((size_t)n_points * 3 * sizeof(double));
    const size_t b_rr = up16((size_t)g.n_dom * sizeof(double));
    const size_t b_dom = on_device ? 0 : up16((size_t)n_points * sizeof(int32_t));
    const size_t need = b_part + b_out + b_pts + b_rr + b_dom;
    if (need > ctx->field_buf_bytes) {
        ctx->dfree(ctx->field_buf);
        ctx->field_buf_bytes = 0;
        ctx->field_buf = ctx->dalloc(need, &rc);
        if (rc) { ctx->field_buf = nullptr; return rc; }
        ctx->field_buf_bytes = need;
    }
    char* buf = (char*)ctx->field_buf;
    float4* part = (float4*)buf;
    double* drr = (double*)(buf + b_part + b_out + b_pts);
    // point arrays on the device
    const double* dp = points;
    const int32_t* dd = domain_of_point;
    double2* dout = (double2*)out;
    if (!on_device) {
        double2* so = (double2*)(buf + b_part);
        double* sp = (double*)(buf + b_part + b_out);
        int32_t* sd = (int32_t*)(buf + b_part + b_out + b_pts + b_rr);
        CK(cudaMemcpyAsync(sp, points, n_points * 3 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(sd, domain_of_point, n_points * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
        dp = sp;
        dd = sd;
        dout = so;
    }
    std::vector<double> rr(g.n_dom);
    for (int j = 0; j < g.n_dom; j++) rr[j] = ctx->doms[j].rho / ctx->rho0;
    CK(cudaMemcpyAsync(drr, rr.data(), g.n_dom * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    FieldArgs a{};
    a.pts = dp; a.dom = dd; a.n = n_points;
    a.pg = ctx->dev.pgp32; a.pd = ctx->dev.pd32; a.tg = ctx->dev.tg32; a.tc = ctx->dev.tc; a.tntri = ctx->dev.tntri;
    a.tdom = ctx->dev.tdom; a.kdom = ctx->dev.kdom; a.rho_ratio = drr; a.k0 = make_double2(ctx->k0re, ctx->k0im);
    a.n_dom = g.n_dom; a.err = ctx->dev.err;
    a.n_tiles = g.n_tiles; a.inc_kind = ctx->field_kind;
    for (int c = 0; c < 3; c++) a.pw_d[c] = ctx->pw_dir[c];
    a.pw_amp = make_double2(ctx->pw_amp[0], ctx->pw_amp[1]);
    a.disc = disc; a.wts = wts; a.n_elem = n_elem; a.nq = nq;
    a.pref = make_double2(0.0, -ctx->omega_rho0 / (2.0 * M_PI));
    a.out = dout;
    a.chunk_tiles = chunk_tiles;
    a.n_chunks = n_chunks;
    a.partial = part;
    CK(launch_field(a, ctx->stream));
    ctx->launches += 3;
    if (!on_device) CK(cudaMemcpyAsync(out, dout, n_points * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return ctx->check_device_error();
}
