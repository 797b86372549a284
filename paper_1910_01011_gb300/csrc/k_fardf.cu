// k_fardf.cu -- the far field (Sec. 2.2 eqs. Form2_matrix_format_p1/_p2, the
// regular-rule part of every operator) to FP64 accuracy in FP32 arithmetic.
//
// GB300 executes FP64 at about 1/64 of its FP32 rate, and an FP64 far-field
// interaction costs ~100 FP64 operations (square root, reciprocal, sincos),
// so the FP64 residual of a matrix-free refinement is ~30x dearer than the
// FP32 operator it corrects.  Here every quantity is a double-float: a pair
// (h, l) of FP32 numbers with |l| <= ulp(h) / 2, about 48 significant bits:
//
//  * sums and products are error-free transformations (Knuth's TwoSum,
//    Dekker's product through a fused multiply-add) written with explicit
//    round-to-nearest intrinsics, so the compiler fuses nothing;
//  * r = |x - y| and 1/r: FP32 square root and reciprocal, then one Newton
//    step each in double-float (relative error ~4e-15);
//  * e^{ikr}: the phase k r is reduced by multiples of pi/64 held in four
//    FP32 parts (Cody and Waite's additive reduction; the first part has 3
//    significant bits, so n (pi/64)_1 is exact for phases below ~100,000 rad),
//    then sin and cos of the remainder |d| <= pi/128 by their Taylor series
//    (the d^3 and d^2 terms in double-float, the rest in FP32) combined with
//    a 128-entry double-float table of sin and cos (j pi/64) by the addition
//    theorem (table-driven method in the manner of Tang);
//  * e^{-Im(k) r} (attenuating domains): reduction by multiples of ln2 / 64,
//    a 64-entry table of 2^(-j/64), Taylor series of the remainder
//    (|t| <= ln2 / 128) and an exact power-of-two scale;
//  * every vector is scaled by a power of two so that its largest density
//    is near 1 (FP32 range), and the sums are (h, l) pairs whose high parts
//    accumulate by TwoSum and whose errors gather in the low parts,
//    renormalised after every source tile (192 terms).
// The tables and split constants are computed on the host in long double.
// Result: the far-field partial potentials of the FP64 path (same layout and
// the same projection), at ~1e-13 relative instead of ~1e-16.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "ctx.h"
#include "df_math.cuh"
#include "internal.h"

namespace gbem {

template <int RG, bool ATTEN>
__device__ __forceinline__ void fardf_body(const FarArgsDF& A, int sl, int grp, const float4* __restrict__ tab,
                                           const float2* __restrict__ etab) {
    const int tid = threadIdx.x;
    const int tt = A.tgt_begin + blockIdx.x;
    const int chunk = blockIdx.y;
    int sb = A.src_begin + chunk * A.chunk_tiles;
    int se = min(sb + A.chunk_tiles, A.src_end);
    const int64_t p = (int64_t)tt * TP + tid;
    const int mt = tid / QP;
    const int mydom = A.tdom[tt];
    if (sl == 1) {
        const int2 dr = A.dom_tiles[mydom];
        sb = max(sb, dr.x);
        se = min(se, dr.y);
    }
    const float4 kk = sl ? A.kdf[mydom] : A.k0df;
    const dfl kr = {kk.x, kk.y}, ki = {kk.z, kk.w};
    const float4 gh = A.pgh[p], gl = A.pgl[p];
    const float4 ch = A.tch[tt], cl = A.tcl[tt];
    const float4 nh = A.tgh[(int64_t)tt * TT + mt], nl = A.tgl[(int64_t)tt * TT + mt];
    const dfl ngx = ld_h(nh, nl, 0), ngy = ld_h(nh, nl, 1), ngz = ld_h(nh, nl, 2);
    const int r0 = grp * RG, nv = min(RG, A.R - r0);
    dfl acc[RG][NCOMP];
#pragma unroll
    for (int v = 0; v < RG; v++)
#pragma unroll
        for (int c = 0; c < NCOMP; c++) acc[v][c] = dfl{0.0f, 0.0f};
    for (int s = sb; s < se; s++) {
        // x - c_source = (x - c_target) + (c_target - c_source)
        const float4 sh = A.tch[s], slo = A.tcl[s];
        const dfl Xx = dadd(ld_h(gh, gl, 0), dsub(ld_h(ch, cl, 0), ld_h(sh, slo, 0)));
        const dfl Xy = dadd(ld_h(gh, gl, 1), dsub(ld_h(ch, cl, 1), ld_h(sh, slo, 1)));
        const dfl Xz = dadd(ld_h(gh, gl, 2), dsub(ld_h(ch, cl, 2), ld_h(sh, slo, 2)));
        const int ntri = A.tntri[s];
        for (int tl = 0; tl < ntri; tl++) {
            if (s == tt && tl == mt) continue;
            const int64_t ts = (int64_t)s * TT + tl;
            const float4 th = A.tgh[ts], tlo = A.tgl[ts];
            const dfl nx = ld_h(th, tlo, 0), ny = ld_h(th, tlo, 1), nz = ld_h(th, tlo, 2);
            const dfl fK = dsub(ld_h(th, tlo, 3), dadd(dadd(dmul(nx, Xx), dmul(ny, Xy)), dmul(nz, Xz)));
            const dfl nn = dadd(dadd(dmul(ngx, nx), dmul(ngy, ny)), dmul(ngz, nz));
            dfl S2r = {0.0f, 0.0f}, S2i = {0.0f, 0.0f};
            for (int q = 0; q < QP; q++) {
                const float4 yh = A.pgh[ts * QP + q], yl = A.pgl[ts * QP + q];
                const dfl ex = dsub(Xx, ld_h(yh, yl, 0)), ey = dsub(Xy, ld_h(yh, yl, 1)), ez = dsub(Xz, ld_h(yh, yl, 2));
                dfl r, ri;
                dsqrt_rinv(dadd(dadd(dsqr(ex), dsqr(ey)), dsqr(ez)), r, ri);
                dfl sn, cs2;
                dsincos(dmul(kr, r), A.c, tab, sn, cs2);
                const dfl a = ATTEN ? dmul(dexp_neg(dmul(ki, r), A.c, etab), ri) : ri;
                const dfl Gr = dmul(a, cs2), Gi = dmul(a, sn);
                const dfl u = dsub(dneg(ki), ri);  // -Im k - 1/r
                const dfl Fr = dmul(dsub(dmul(Gr, u), dmul(Gi, kr)), ri);
                const dfl Fi = dmul(dadd(dmul(Gr, kr), dmul(Gi, u)), ri);
                const dfl ndot = dadd(dadd(dmul(ngx, ex), dmul(ngy, ey)), dmul(ngz, ez));
                const dfl nFr = dmul(ndot, Fr), nFi = dmul(ndot, Fi);  // K' point factor
                const dfl kFr = dmul(fK, Fr), kFi = dmul(fK, Fi);      // K point factor
                const dfl wGr = dmul(nn, Gr), wGi = dmul(nn, Gi);      // W (normal-normal) point factor
                const dfl w = ld_h(yh, yl, 3);
                dmac(S2r, Gr, w, 1.0f);
                dmac(S2i, Gi, w, 1.0f);
#pragma unroll
                for (int v = 0; v < RG; v++) {
                    if (v >= nv) break;
                    const int64_t i = (int64_t)(r0 + v) * A.n_pts + ts * QP + q;
                    const float4 dh = A.pdh[i], dl = A.pdl[i];
                    const dfl dx = ld_h(dh, dl, 0), dy = ld_h(dh, dl, 1), dz = ld_h(dh, dl, 2), dw = ld_h(dh, dl, 3);
                    dmac(acc[v][0], Gr, dx, 1.0f);
                    dmac(acc[v][0], Gi, dy, -1.0f);
                    dmac(acc[v][1], Gr, dy, 1.0f);
                    dmac(acc[v][1], Gi, dx, 1.0f);
                    dmac(acc[v][2], kFr, dz, 1.0f);
                    dmac(acc[v][2], kFi, dw, -1.0f);
                    dmac(acc[v][3], kFr, dw, 1.0f);
                    dmac(acc[v][3], kFi, dz, 1.0f);
                    dmac(acc[v][4], nFr, dx, 1.0f);
                    dmac(acc[v][4], nFi, dy, -1.0f);
                    dmac(acc[v][5], nFr, dy, 1.0f);
                    dmac(acc[v][5], nFi, dx, 1.0f);
                    dmac(acc[v][6], wGr, dz, 1.0f);
                    dmac(acc[v][6], wGi, dw, -1.0f);
                    dmac(acc[v][7], wGr, dw, 1.0f);
                    dmac(acc[v][7], wGi, dz, 1.0f);
                }
            }
#pragma unroll
            for (int v = 0; v < RG; v++) {
                if (v >= nv) break;
                const int64_t i = (int64_t)(r0 + v) * 2 * A.n_slots + 2 * ts;
                const float4 reh = A.cuh[i], rel = A.cul[i], imh = A.cuh[i + 1], iml = A.cul[i + 1];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    const dfl cre = ld_h(reh, rel, c), cim = ld_h(imh, iml, c);
                    dmac(acc[v][8 + c], S2r, cre, 1.0f);
                    dmac(acc[v][8 + c], S2i, cim, -1.0f);
                    dmac(acc[v][11 + c], S2r, cim, 1.0f);
                    dmac(acc[v][11 + c], S2i, cre, 1.0f);
                }
            }
        }
        // renormalise after every source tile: the low parts stay below half an
        // ulp of the high parts, so their own rounding does not grow with the chunk
#pragma unroll
        for (int v = 0; v < RG; v++)
#pragma unroll
            for (int c = 0; c < NCOMP; c++) acc[v][c] = two_sum(acc[v][c].h, acc[v][c].l);
    }
#pragma unroll
    for (int v = 0; v < RG; v++) {
        if (v >= nv) break;
        const double scale = ldexp(1.0, A.vexp[r0 + v]);
        double* out = A.partial + (int64_t)(r0 + v) * A.rstride + ((int64_t)chunk * 2 + sl) * NCOMP * A.n_pts + p;
#pragma unroll
        for (int c = 0; c < NCOMP; c++) out[(int64_t)c * A.n_pts] = ((double)acc[v][c].h + (double)acc[v][c].l) * scale;
    }
}

template <int RG>
__global__ void __launch_bounds__(TP, RG == 1 ? 2 : 1) fardf_kernel(FarArgsDF A) {
    __shared__ float4 tab[128];
    __shared__ float2 etab[64];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) tab[i] = A.sctab[i];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) etab[i] = A.extab[i];
    __syncthreads();
    const int sl = blockIdx.z / A.groups, grp = blockIdx.z % A.groups;
    const float4 kk = sl ? A.kdf[A.tdom[A.tgt_begin + blockIdx.x]] : A.k0df;
    if (kk.z != 0.0f || kk.w != 0.0f) fardf_body<RG, true>(A, sl, grp, tab, etab);
    else fardf_body<RG, false>(A, sl, grp, tab, etab);
}

// ----------------------------------------------------------------- splitting

// hi = fl32(v s), lo = fl32(v s - hi) component-wise, s = 2^-e (e from *ebits, or 0)
__global__ void df_split4_kernel(const double4* __restrict__ v, int64_t n, int64_t per_vec, const int* __restrict__ vexp,
                                 float4* __restrict__ hi, float4* __restrict__ lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = vexp ? ldexp(1.0, -vexp[i / per_vec]) : 1.0;
    const double4 x = v[i];
    const double c[4] = {x.x * s, x.y * s, x.z * s, x.w * s};
    float h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        h[k] = (float)c[k];
        l[k] = (float)(c[k] - (double)h[k]);
    }
    hi[i] = make_float4(h[0], h[1], h[2], h[3]);
    lo[i] = make_float4(l[0], l[1], l[2], l[3]);
}

// largest |component| over each vector's densities and curls, as ordered bits
__global__ void df_vmax_kernel(const double4* __restrict__ pd, int64_t n_pts, const double4* __restrict__ cu,
                               int64_t n_cu, unsigned long long* __restrict__ out) {
    const int r = blockIdx.y;
    unsigned long long m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pts + n_cu;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double4 x = i < n_pts ? pd[(int64_t)r * n_pts + i] : cu[(int64_t)r * n_cu + (i - n_pts)];
        const double a = fmax(fmax(fabs(x.x), fabs(x.y)), fmax(fabs(x.z), fabs(x.w)));
        const unsigned long long b = (unsigned long long)__double_as_longlong(a);
        m = b > m ? b : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&out[r], m);
}

// exponent e with max = f 2^e, f in [1/2, 1) (0 for zero or non-finite)
__global__ void df_vexp_kernel(const unsigned long long* __restrict__ bits, int R, int* __restrict__ vexp) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double m = __longlong_as_double((long long)bits[r]);
    int e = 0;
    if (m > 0 && isfinite(m)) frexp(m, &e);
    vexp[r] = e;
}

}  // namespace gbem

using namespace gbem;

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

namespace {

// (h, l) of a long double
void split_ld(long double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (long double)h);
}

// v rounded to `bits` significant bits (so that n v is exact in FP32 for n < 2^(24 - bits))
float round_bits(long double v, int bits) {
    int e;
    const long double f = std::frexp(v, &e);
    return (float)std::ldexp(std::round(std::ldexp(f, bits)), e - bits);
}

}  // namespace

// Largest phase |Re k| |x - y| the double-float reduction handles (n (pi/64)_1
// exact for n < 2^21), with a margin.
constexpr double DF_PHASE_MAX = 1.0e5;

// Extent of the mesh (and of the transducer's pistons if `with_transducer`):
// the diagonal of the box around every tile's bounding sphere.
double bem_ctx::df_extent(bool with_transducer) const {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int t = 0; t < geo.n_tiles; t++)
        for (int c = 0; c < 3; c++) {
            lo[c] = std::min(lo[c], geo.tile_c[4 * t + c] - geo.tile_c[4 * t + 3]);
            hi[c] = std::max(hi[c], geo.tile_c[4 * t + c] + geo.tile_c[4 * t + 3]);
        }
    if (with_transducer)
        for (size_t m = 0; m < tr_r.size(); m++)
            for (int c = 0; c < 3; c++) {
                lo[c] = std::min(lo[c], tr_c[3 * m + c] - tr_r[m]);
                hi[c] = std::max(hi[c], tr_c[3 * m + c] + tr_r[m]);
            }
    double d2 = 0;
    for (int c = 0; c < 3; c++) d2 += hi[c] > lo[c] ? (hi[c] - lo[c]) * (hi[c] - lo[c]) : 0.0;
    return std::sqrt(d2);
}

// INVALID_ARG if a phase |Re k| |x - y| of this geometry (wavenumber kre, the
// domains' own, and the exterior one) may exceed the double-float range.
int bem_ctx::check_df_phase(double kre, bool with_transducer) {
    double kmax = std::max(std::fabs(kre), std::fabs(k0re));
    for (auto& d : doms) kmax = std::max(kmax, std::fabs(d.kre));
    if (kmax * df_extent(with_transducer) > DF_PHASE_MAX)
        return fail(BEM_ERR_INVALID_ARG, "phases k|x - y| beyond the double-float range (1e5 rad): set "
                                         "bem_opts.fp64_far = 1 for native FP64 arithmetic");
    return BEM_OK;
}

// Geometry, tables and constants of the double-float far field (once per geometry).
int bem_ctx::ensure_fardf() {
    bem_ctx* const ctx = this;
    if (dfg.ready) return BEM_OK;
    const Geometry& g = geo;
    int rc;
    const int64_t np = g.n_pts, ns = g.n_slots, nt = g.n_tiles;
    const size_t bytes = (size_t)2 * (np + ns + nt) * sizeof(float4) + 128 * sizeof(float4) + 64 * sizeof(float2) +
                         (size_t)g.n_dom * sizeof(float4);
    dfg.buf = dalloc(bytes, &rc);
    if (rc) { dfg.buf = nullptr; return rc; }
    float4* f = (float4*)dfg.buf;
    dfg.pgh = f; dfg.pgl = f + np; f += 2 * np;
    dfg.tgh = f; dfg.tgl = f + ns; f += 2 * ns;
    dfg.tch = f; dfg.tcl = f + nt; f += 2 * nt;
    dfg.sctab = f; f += 128;
    dfg.kdf = f; f += g.n_dom;
    dfg.extab = (float2*)f;
    auto split = [&](const double4* src, int64_t n, float4* h, float4* l) -> int {
        if (n <= 0) return BEM_OK;
        df_split4_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(src, n, n, nullptr, h, l);
        launches += 1;
        return cudaGetLastError() == cudaSuccess ? BEM_OK : BEM_ERR_CUDA;
    };
    if ((rc = split(dev.pg64, np, dfg.pgh, dfg.pgl)) || (rc = split(dev.tg64, ns, dfg.tgh, dfg.tgl)) ||
        (rc = split(dev.tc, nt, dfg.tch, dfg.tcl)))
        return fail(rc, "double-float geometry split");
    const long double PI = 3.141592653589793238462643383279502884L, LN2 = 0.693147180559945309417232121458176568L;
    std::vector<float4> sc(128);
    for (int j = 0; j < 128; j++) {
        const long double a = (long double)j * PI / 64.0L;
        split_ld(std::sin(a), sc[j].x, sc[j].y);
        split_ld(std::cos(a), sc[j].z, sc[j].w);
    }
    std::vector<float2> ex(64);
    for (int j = 0; j < 64; j++) split_ld(std::exp2(-(long double)j / 64.0L), ex[j].x, ex[j].y);
    std::vector<float4> kd(g.n_dom);
    for (int d = 0; d < g.n_dom; d++) {
        split_ld((long double)doms[d].kre, kd[d].x, kd[d].y);
        split_ld((long double)doms[d].kim, kd[d].z, kd[d].w);
    }
    CK(cudaMemcpyAsync(dfg.sctab, sc.data(), sc.size() * sizeof(float4), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(dfg.extab, ex.data(), ex.size() * sizeof(float2), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(dfg.kdf, kd.data(), kd.size() * sizeof(float4), cudaMemcpyHostToDevice, stream));
    // pi/64 in four parts (the first with 3 significant bits), ln2/64 in three (the first with 10)
    DfConsts& c = dfg.c;
    long double rest = PI / 64.0L;
    c.pi64[0] = round_bits(rest, 3);
    rest -= c.pi64[0];
    for (int i = 1; i < 4; i++) {
        c.pi64[i] = (float)rest;
        rest -= c.pi64[i];
    }
    rest = LN2 / 64.0L;
    c.ln64[0] = round_bits(rest, 10);
    rest -= c.ln64[0];
    for (int i = 1; i < 3; i++) {
        c.ln64[i] = (float)rest;
        rest -= c.ln64[i];
    }
    c.inv_pi64 = (float)(64.0L / PI);
    c.inv_ln64 = (float)(64.0L / LN2);
    split_ld(-1.0L / 6.0L, c.sixth[0], c.sixth[1]);
    CK(cudaStreamSynchronize(stream));  // the host tables above are freed on return
    dfg.ready = true;
    return BEM_OK;
}

// Partial potentials of R vectors whose densities pd [R][n_pts] and curls
// cu [R][2 n_slots] (FP64, from the gather) are given: the double-float far
// field over target tiles [tgt_b, tgt_e) and source tiles [src_b, src_e),
// into partial [R][n_chunks][2][NCOMP][n_pts] (rstride doubles apart).
int bem_ctx::far_df(const double4* pd, const double4* cu, int64_t R, int tgt_b, int tgt_e, int src_b, int src_e,
                    int chunk_tiles, int n_chunks, int slot1, double kre, double kim, double* partial,
                    int64_t rstride) {
    bem_ctx* const ctx = this;
    int rc = ensure_fardf();
    if (!rc) rc = check_df_phase(kre, false);
    if (rc) return rc;
    const Geometry& g = geo;
    const int64_t np = g.n_pts, ns2 = 2 * g.n_slots;
    const size_t need = (size_t)R * 2 * (np + ns2) * sizeof(float4) + (size_t)R * (sizeof(int) + 8);
    if (need > dfv_bytes) {
        dfree(dfv_buf);
        dfv_buf = dalloc(need, &rc);
        if (rc) { dfv_buf = nullptr; dfv_bytes = 0; return rc; }
        dfv_bytes = need;
    }
    float4* f = (float4*)dfv_buf;
    float4 *pdh = f, *pdl = f + R * np;
    f += 2 * R * np;
    float4 *cuh = f, *cul = f + R * ns2;
    f += 2 * R * ns2;
    unsigned long long* mb = (unsigned long long*)f;
    int* vexp = (int*)(mb + R);
    CK(cudaMemsetAsync(mb, 0, R * sizeof(unsigned long long), stream));
    const int nbx = (int)std::min<int64_t>(1024, (np + ns2 + 255) / 256);
    df_vmax_kernel<<<dim3((unsigned)nbx, (unsigned)R), 256, 0, stream>>>(pd, np, cu, ns2, mb);
    df_vexp_kernel<<<(unsigned)((R + 127) / 128), 128, 0, stream>>>(mb, (int)R, vexp);
    df_split4_kernel<<<(unsigned)((R * np + 255) / 256), 256, 0, stream>>>(pd, R * np, np, vexp, pdh, pdl);
    df_split4_kernel<<<(unsigned)((R * ns2 + 255) / 256), 256, 0, stream>>>(cu, R * ns2, ns2, vexp, cuh, cul);
    launches += 4;
    FarArgsDF a{};
    a.pgh = dfg.pgh; a.pgl = dfg.pgl; a.tgh = dfg.tgh; a.tgl = dfg.tgl; a.tch = dfg.tch; a.tcl = dfg.tcl;
    a.tdom = dev.tdom; a.tntri = dev.tntri; a.dom_tiles = dev.dom_tiles; a.kdf = dfg.kdf;
    float kh, kl, ih, il;
    split_ld((long double)kre, kh, kl);
    split_ld((long double)kim, ih, il);
    a.k0df = make_float4(kh, kl, ih, il);
    a.pdh = pdh; a.pdl = pdl; a.cuh = cuh; a.cul = cul; a.vexp = vexp;
    a.sctab = dfg.sctab; a.extab = dfg.extab;
    a.c = dfg.c;
    a.src_begin = src_b; a.src_end = src_e; a.tgt_begin = tgt_b; a.chunk_tiles = chunk_tiles; a.slot1 = slot1;
    a.R = (int)R; a.groups = R == 1 ? 1 : (int)((R + RG64 - 1) / RG64);
    a.n_pts = np; a.n_slots = g.n_slots; a.rstride = rstride; a.partial = partial;
    const int n_tgt = tgt_e - tgt_b;
    if (n_tgt <= 0 || n_chunks <= 0) return BEM_OK;
    const dim3 grid((unsigned)n_tgt, (unsigned)n_chunks, (unsigned)((slot1 ? 2 : 1) * a.groups));
    if (R == 1) fardf_kernel<1><<<grid, TP, 0, stream>>>(a);
    else fardf_kernel<RG64><<<grid, TP, 0, stream>>>(a);
    launches += 1;
    CK(cudaGetLastError());
    return BEM_OK;
}
