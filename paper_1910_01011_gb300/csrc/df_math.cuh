// df_math.cuh -- double-float arithmetic (a real as a pair (h, l) of FP32
// numbers, |l| <= ulp(h) / 2, about 48 significant bits) for the FP64-accurate
// kernels that run on the FP32 pipes (k_fardf.cu, the piston right-hand
// sides in bem_solve.cu).  Sums and products are error-free transformations
// (Knuth's TwoSum; Dekker's product through a fused multiply-add) written with
// explicit round-to-nearest intrinsics, so the compiler fuses nothing.
//  * dsqrt_rinv: FP32 square root and reciprocal, one Newton step each.
//  * dsincos: Cody and Waite's additive reduction of the phase by multiples of
//    pi/64 held in four FP32 parts (the first with 3 significant bits, so its
//    product with the multiple n is exact for n < 2^21, phases below ~100,000
//    rad; the next two products are formed exactly), Taylor series of the remainder
//    |d| <= pi/128 (d^3 and d^2 terms in double-float, the rest in FP32), and
//    a 128-entry double-float table of sin, cos (j pi/64) combined by the
//    addition theorem (table-driven method in the manner of Tang).
//  * dexp_neg: e^{-a} by reduction with ln2/64, a 64-entry table of
//    2^(-j/64), the Taylor series of the remainder (|t| <= ln2/128) and an
//    exact power-of-two scale.
// The tables and split constants (DfConsts) are computed on the host in long
// double (bem_ctx::ensure_fardf).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace gbem {

struct dfl {
    float h, l;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ dfl dneg(dfl a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dfl dadd(dfl a, dfl b) {
    const dfl s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dfl dsub(dfl a, dfl b) { return dadd(a, dneg(b)); }
__device__ __forceinline__ dfl dmul(dfl a, dfl b) {
    const dfl p = two_prod(a.h, b.h);
    return fast_two_sum(p.h, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l)));
}
__device__ __forceinline__ dfl dsqr(dfl a) {
    const dfl p = two_prod(a.h, a.h);
    return fast_two_sum(p.h, __fmaf_rn(__fadd_rn(a.h, a.h), a.l, p.l));
}
// acc += s a b (s = +-1); acc's low part gathers the errors (renormalised at the end)
__device__ __forceinline__ void dmac(dfl& acc, dfl a, dfl b, float s) {
    const dfl p = two_prod(s * a.h, b.h);
    const float t = __fmaf_rn(s * a.h, b.l, __fmaf_rn(s * a.l, b.h, p.l));
    const dfl q = two_sum(acc.h, p.h);
    acc.h = q.h;
    acc.l = __fadd_rn(acc.l, __fadd_rn(q.l, t));
}

__device__ __forceinline__ dfl ld_h(const float4& h, const float4& l, int c) {
    return c == 0 ? dfl{h.x, l.x} : c == 1 ? dfl{h.y, l.y} : c == 2 ? dfl{h.z, l.z} : dfl{h.w, l.w};
}

// r = sqrt(R) and 1/r for R > 0 (double-float): FP32 seeds, one Newton step each
__device__ __forceinline__ void dsqrt_rinv(dfl R, dfl& r, dfl& ri) {
    const float s = __fsqrt_rn(R.h);
    const float y = __frcp_rn(s);
    const dfl s2 = two_prod(s, s);
    const float d = __fadd_rn(__fsub_rn(R.h, s2.h), __fsub_rn(R.l, s2.l));  // R - s^2 (first difference exact)
    r = fast_two_sum(s, __fmul_rn(__fmul_rn(d, y), 0.5f));
    const dfl ry = two_prod(r.h, y);
    const float e = __fsub_rn(__fsub_rn(1.0f, ry.h), __fmaf_rn(r.l, y, ry.l));  // 1 - r y
    ri = fast_two_sum(y, __fmul_rn(y, e));
}

// sin and cos of th >= 0 (double-float) by reduction to |d| <= pi/128
__device__ __forceinline__ void dsincos(dfl th, const DfConsts& A, const float4* __restrict__ tab, dfl& sn, dfl& cs) {
    const float nf = rintf(__fmul_rn(th.h, A.inv_pi64));
    const float r1 = __fsub_rn(th.h, __fmul_rn(nf, A.pi64[0]));  // exact (n (pi/64)_1 is exact and near th)
    const dfl p2 = two_prod(nf, A.pi64[1]);                       // n (pi/64)_2 and n (pi/64)_3 exactly
    const dfl p3 = two_prod(nf, A.pi64[2]);
    const dfl s = two_sum(r1, -p2.h);
    const dfl t = two_sum(s.h, -p3.h);
    float lo = __fsub_rn(__fsub_rn(s.l, p2.l), p3.l);
    lo = __fadd_rn(lo, t.l);
    lo = __fmaf_rn(-nf, A.pi64[3], lo);
    lo = __fadd_rn(lo, th.l);
    const dfl d = two_sum(t.h, lo);
    const float4 ta = tab[((int)nf) & 127];
    const dfl sa = {ta.x, ta.y}, ca = {ta.z, ta.w};
    const dfl d2 = dsqr(d);
    // sin d = d - d^3 / 6 + d^5 / 120 - d^7 / 5040
    const dfl d3 = dmul(d, d2);
    dfl sd = dadd(d, dmul(d3, dfl{A.sixth[0], A.sixth[1]}));
    sd.l = __fmaf_rn(__fmul_rn(d3.h, d2.h), __fmaf_rn(-d2.h, 1.0f / 5040.0f, 1.0f / 120.0f), sd.l);
    // cos d = 1 - d^2 / 2 + d^4 / 24 - d^6 / 720
    dfl cd = fast_two_sum(1.0f, -0.5f * d2.h);
    cd.l = __fmaf_rn(__fmul_rn(d2.h, d2.h), __fmaf_rn(-d2.h, 1.0f / 720.0f, 1.0f / 24.0f), __fsub_rn(cd.l, 0.5f * d2.l));
    sn = dadd(dmul(sa, cd), dmul(ca, sd));
    cs = dsub(dmul(ca, cd), dmul(sa, sd));
}

// e^{-a} (double-float) by reduction to |t| <= ln2 / 128
__device__ __forceinline__ dfl dexp_neg(dfl a, const DfConsts& A, const float2* __restrict__ etab) {
    const float mf = rintf(__fmul_rn(a.h, A.inv_ln64));
    const float r1 = __fsub_rn(a.h, __fmul_rn(mf, A.ln64[0]));
    const dfl p2 = two_prod(mf, A.ln64[1]);
    const dfl s = two_sum(r1, -p2.h);
    float lo = __fsub_rn(s.l, p2.l);
    lo = __fmaf_rn(-mf, A.ln64[2], lo);
    lo = __fadd_rn(lo, a.l);
    const dfl t = fast_two_sum(s.h, lo);
    // e^{-t} = 1 - t + t^2 / 2 - t^3 / 6 + t^4 / 24
    const dfl t2 = dsqr(t);
    dfl e = dadd(dsub(dfl{1.0f, 0.0f}, t), dfl{0.5f * t2.h, 0.5f * t2.l});
    e.l = __fmaf_rn(__fmul_rn(t.h, t2.h), __fmaf_rn(t.h, 1.0f / 24.0f, -1.0f / 6.0f), e.l);
    const int m = (int)mf;
    const float2 T = etab[m & 63];
    const int k = m >> 6;  // 2^(-m/64) = 2^(-k) 2^(-(m & 63)/64)
    if (k > 126) return {0.0f, 0.0f};
    const float sc = __int_as_float((127 - k) << 23);
    const dfl v = dmul(e, dfl{T.x, T.y});
    return {v.h * sc, v.l * sc};
}

}  // namespace gbem
