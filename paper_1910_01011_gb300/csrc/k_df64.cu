// k_df64.cu -- complex products to FP64 accuracy in FP32 arithmetic.
//
// The FP64 residual of the refinement (r = b - A_hat u with the complex128
// A_hat) and the excitation superposition (u = w x basis) are matrix products
// whose operand is read once.  GB300 executes FP64 at about 1/64 of its FP32
// rate, so the same products in FP64 arithmetic are bound by that rate (8 N^2
// FP64 flops per vector: ~11 ms on a 41k-unknown A_hat) rather than by
// reading the 16 N^2 bytes (~4 ms).  Here every matrix entry is stored as a
// pair of FP32 numbers in the same 16 bytes, and the products and sums are
// carried out with error-free FP32 transformations:
//
//  * storage (set-up): the matrix is scaled by 2^-e so that its largest
//    entry lies in [1/2, 1), and each scaled FP64 part v becomes
//    hi = fl32(v), lo = fl32(v - hi), |v - hi - lo| <= 2^-48 |v|; a float4
//    per entry holds (hi re, hi im, lo re, lo im).  Vectors are split the
//    same way per call, each right-hand side with its own power of two.
//  * products: hi_a hi_x is formed exactly as p + fma(hi_a, hi_x, -p)
//    (Dekker's product with a fused multiply-add); the cross terms
//    hi_a lo_x + lo_a hi_x are ~2^-24 of it and go into the low part with
//    ordinary FMAs; lo_a lo_x (~2^-48) is dropped.
//  * sums: the high parts are accumulated with Knuth's TwoSum, whose
//    rounding error is exact and goes into the low accumulator; every 256
//    terms a lane folds its (high, low) pair into FP64, and at the end the
//    32 lanes of a warp are summed in FP64.
//
// Real and imaginary parts of an output are the two lanes of one packed
// FP32 value (FFMA2 / FADD2 / FMUL2), so y += a x for complex a, x is
//   (y_re, y_im) += x_re (a_re, a_im) + x_im (-a_im, a_re).
// A float32 emulation of this order of operations on 41,320-term rows with
// oscillating, decaying entries gives a relative l2 error of 1.1e-13 against
// extended-precision sums (5.9e-13 without the FP64 folds).
#include <cuda_runtime.h>

#include <cstdint>

#include "ctx.h"
#include "internal.h"
#include "pair_math.h"

namespace gbem {

constexpr int DF_WARPS = 8;    // warps per CTA
constexpr int DF_FOLD = 256;   // terms a lane accumulates in FP32 between FP64 folds

// ----------------------------------------------------------------- splitting

// Largest |re|, |im| of n complex values, as the bit pattern of a
// non-negative double (these order like integers), max-ed into out[seg] for
// the segment seg = index / seg_len.
__global__ void df_maxbits_kernel(const double2* __restrict__ v, int64_t n, int64_t seg_len,
                                  unsigned long long* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long m = 0;
    int64_t seg = i < n ? i / seg_len : -1;
    for (; i < n; i += stride) {
        const int64_t s = i / seg_len;
        if (s != seg) {
            if (m) atomicMax(&out[seg], m);
            m = 0;
            seg = s;
        }
        const double2 x = v[i];
        const unsigned long long b = (unsigned long long)__double_as_longlong(fmax(fabs(x.x), fabs(x.y)));
        m = b > m ? b : m;
    }
    if (seg >= 0 && m) atomicMax(&out[seg], m);
}

// Exponent e with max = f 2^e, f in [1/2, 1) (0 for a zero or non-finite max).
__device__ __forceinline__ int df_exponent(unsigned long long bits) {
    const double m = __longlong_as_double((long long)bits);
    if (!(m > 0) || !isfinite(m)) return 0;
    int e;
    frexp(m, &e);
    return e;
}

__device__ __forceinline__ float4 df_split(double2 v, double scale) {
    const double re = v.x * scale, im = v.y * scale;
    const float hr = (float)re, hi = (float)im;
    return make_float4(hr, hi, (float)(re - (double)hr), (float)(im - (double)hi));
}

// In place: complex128 entries -> scaled FP32 (hi, lo) pairs (same 16 bytes).
__global__ void df_split_inplace_kernel(double2* v, int64_t n, const unsigned long long* __restrict__ maxbits,
                                        int* __restrict__ e_out) {
    const int e = df_exponent(maxbits[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0) *e_out = e;
    const double scale = ldexp(1.0, -e);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double2 x = v[i];
        reinterpret_cast<float4*>(v)[i] = df_split(x, scale);
    }
}

// R vectors of seg_len complex128 values -> split copies, each vector with
// its own exponent (e_out[r]).
__global__ void df_split_vectors_kernel(const double2* __restrict__ x, int64_t seg_len, int64_t R,
                                        const unsigned long long* __restrict__ maxbits, float4* __restrict__ out,
                                        int* __restrict__ e_out) {
    const int64_t n = seg_len * R;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t r = i / seg_len;
        const int e = df_exponent(maxbits[r]);
        if (i == r * seg_len) e_out[r] = e;
        out[i] = df_split(x[i], ldexp(1.0, -e));
    }
}

// ----------------------------------------------------------------- accumulation

struct DfAcc {
    f2 S, L;  // high parts (TwoSum) and low parts, lanes (re, im)
};

__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return add2(a, neg2(b)); }

// s + p = s' + e exactly (Knuth's TwoSum, per lane); e is added to L.
__device__ __forceinline__ void two_sum_into(DfAcc& c, f2 p) {
    const f2 t = add2(c.S, p);
    const f2 bb = sub2(t, c.S);
    const f2 e = add2(sub2(c.S, sub2(t, bb)), sub2(p, bb));
    c.S = t;
    c.L = add2(c.L, e);
}

// c += a x for one matrix entry a (hi, lo in A = (hr, hi), AS = (-hi, hr),
// AL, ALS likewise) and one split vector entry x = (hr, hi, lr, li).
__device__ __forceinline__ void df_mac(DfAcc& c, f2 A, f2 AS, f2 AL, f2 ALS, const float4& x) {
    const f2 xr = bc2(x.x), xi = bc2(x.y);
    const f2 P = mul2(A, xr), Q = mul2(AS, xi);
    const f2 Pe = fma2(A, xr, neg2(P)), Qe = fma2(AS, xi, neg2(Q));  // exact product errors
    two_sum_into(c, P);
    two_sum_into(c, Q);
    const f2 cross = fma2(AL, xr, fma2(ALS, xi, fma2(A, bc2(x.z), fma2(AS, bc2(x.w), add2(Pe, Qe)))));
    c.L = add2(c.L, cross);
}

__device__ __forceinline__ void df_fold(DfAcc& c, double2& acc) {
    acc.x += (double)c.S.x + (double)c.L.x;
    acc.y += (double)c.S.y + (double)c.L.y;
    c.S = make_float2(0.f, 0.f);
    c.L = make_float2(0.f, 0.f);
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// ----------------------------------------------------------------- Y = X A^T (rows of A reduced)

struct DfGemvArgs {
    const float4* A;      // [m][lda] split entries, scaled by 2^-eA
    int64_t m, k, lda;
    const int* eA;        // device scalar
    const float4* X;      // [R][k] split vectors
    const int* eX;        // [R]
    int64_t R;
    double2* Y;           // [R][ldy]
    int64_t ldy;
};

// One warp per RW rows of A; lanes stride over the k columns (coalesced
// 16-byte loads); right-hand sides in groups of RG, each group one pass over
// the warp's rows.
template <int RW, int RG>
__global__ void __launch_bounds__(DF_WARPS * 32) df_gemv_kernel(DfGemvArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t n_groups = (a.m + RW - 1) / RW;
    const int eA = *a.eA;
    for (int64_t g = (int64_t)blockIdx.x * DF_WARPS + (threadIdx.x >> 5); g < n_groups;
         g += (int64_t)gridDim.x * DF_WARPS) {
        const int64_t i0 = g * RW;
        const float4* Arow[RW];
#pragma unroll
        for (int w = 0; w < RW; w++) Arow[w] = a.A + min(i0 + w, a.m - 1) * a.lda;
        for (int64_t r0 = 0; r0 < a.R; r0 += RG) {
            const float4* Xr[RG];
#pragma unroll
            for (int q = 0; q < RG; q++) Xr[q] = a.X + min(r0 + q, a.R - 1) * a.k;
            DfAcc c[RW][RG];
            double2 acc[RW][RG];
#pragma unroll
            for (int w = 0; w < RW; w++)
#pragma unroll
                for (int q = 0; q < RG; q++) {
                    c[w][q].S = c[w][q].L = make_float2(0.f, 0.f);
                    acc[w][q] = make_double2(0.0, 0.0);
                }
            for (int64_t jb = 0; jb < a.k; jb += 32 * DF_FOLD) {
                const int64_t je = min(a.k, jb + 32 * DF_FOLD);
#pragma unroll 2
                for (int64_t j = jb + lane; j < je; j += 32) {
                    float4 xv[RG];
#pragma unroll
                    for (int q = 0; q < RG; q++) xv[q] = __ldg(Xr[q] + j);
#pragma unroll
                    for (int w = 0; w < RW; w++) {
                        const float4 av = __ldcs(Arow[w] + j);  // streamed: each entry is read once per pass
                        const f2 A = make_float2(av.x, av.y), AS = make_float2(-av.y, av.x);
                        const f2 AL = make_float2(av.z, av.w), ALS = make_float2(-av.w, av.z);
#pragma unroll
                        for (int q = 0; q < RG; q++) df_mac(c[w][q], A, AS, AL, ALS, xv[q]);
                    }
                }
#pragma unroll
                for (int w = 0; w < RW; w++)
#pragma unroll
                    for (int q = 0; q < RG; q++) df_fold(c[w][q], acc[w][q]);
            }
#pragma unroll
            for (int w = 0; w < RW; w++)
#pragma unroll
                for (int q = 0; q < RG; q++) {
                    const double2 s = warp_sum(acc[w][q]);
                    if (lane == 0 && i0 + w < a.m && r0 + q < a.R) {
                        const int e = eA + a.eX[r0 + q];
                        a.Y[(r0 + q) * a.ldy + i0 + w] = make_double2(ldexp(s.x, e), ldexp(s.y, e));
                    }
                }
        }
    }
}

// ----------------------------------------------------------------- U = W B (rows of B combined)

struct DfCombineArgs {
    const float4* B;      // [K][n] split rows, scaled by 2^-eB
    int64_t K, n;
    const int* eB;
    const float4* W;      // [R][K] split weights
    const int* eW;        // [R]
    int64_t R;
    double2* U;           // [R][n]
};

// One thread per column j (coalesced across the warp), RG outputs at a time;
// the weights of a row are the same for every thread (broadcast loads).
template <int RG>
__global__ void __launch_bounds__(256) df_combine_kernel(DfCombineArgs a) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * RG;
    if (j >= a.n) return;
    const int eB = *a.eB;
    DfAcc c[RG];
    double2 acc[RG];
#pragma unroll
    for (int q = 0; q < RG; q++) {
        c[q].S = c[q].L = make_float2(0.f, 0.f);
        acc[q] = make_double2(0.0, 0.0);
    }
    for (int64_t m0 = 0; m0 < a.K; m0 += DF_FOLD) {
        const int64_t m1 = min(a.K, m0 + DF_FOLD);
        for (int64_t m = m0; m < m1; m++) {
            const float4 bv = __ldcs(a.B + m * a.n + j);
            const f2 A = make_float2(bv.x, bv.y), AS = make_float2(-bv.y, bv.x);
            const f2 AL = make_float2(bv.z, bv.w), ALS = make_float2(-bv.w, bv.z);
#pragma unroll
            for (int q = 0; q < RG; q++) {
                const float4 wv = __ldg(a.W + min(r0 + q, a.R - 1) * a.K + m);
                df_mac(c[q], A, AS, AL, ALS, wv);
            }
        }
#pragma unroll
        for (int q = 0; q < RG; q++) df_fold(c[q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < RG; q++)
        if (r0 + q < a.R) {
            const int e = eB + a.eW[r0 + q];
            a.U[(r0 + q) * a.n + j] = make_double2(ldexp(acc[q].x, e), ldexp(acc[q].y, e));
        }
}

// ----------------------------------------------------------------- host side

namespace {

// Scratch of one call: exponents and max bits of R vectors, the split copies.
struct DfScratch {
    unsigned long long* maxbits;
    int* e;
    float4* xs;
};

int df_scratch(bem_ctx* ctx, int64_t R, int64_t len, DfScratch* s) {
    const size_t need = (size_t)R * (sizeof(unsigned long long) + sizeof(int)) + 256 + (size_t)R * len * sizeof(float4);
    if (need > ctx->df_work_bytes) {
        ctx->dfree(ctx->df_work);
        int rc;
        ctx->df_work = ctx->dalloc(need, &rc);
        if (rc) {
            ctx->df_work = nullptr;
            ctx->df_work_bytes = 0;
            return rc;
        }
        ctx->df_work_bytes = need;
    }
    char* p = (char*)ctx->df_work;
    s->xs = (float4*)p;  // 16-byte aligned at the start of the allocation
    p += (size_t)R * len * sizeof(float4);
    s->maxbits = (unsigned long long*)p;
    s->e = (int*)(p + (size_t)R * sizeof(unsigned long long));
    return BEM_OK;
}

unsigned grid_for(int64_t n, int threads) { return (unsigned)std::min<int64_t>((n + threads - 1) / threads, 152 * 16); }

// Split R vectors x [R][len] into s->xs with one exponent per vector.
int split_vectors(bem_ctx* ctx, const double2* x, int64_t R, int64_t len, DfScratch* s) {
    int rc = df_scratch(ctx, R, len, s);
    if (rc) return rc;
    cudaError_t e = cudaMemsetAsync(s->maxbits, 0, R * sizeof(unsigned long long), ctx->stream);
    if (e != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string("df split: ") + cudaGetErrorString(e));
    df_maxbits_kernel<<<grid_for(R * len, 256), 256, 0, ctx->stream>>>(x, R * len, len, s->maxbits);
    df_split_vectors_kernel<<<grid_for(R * len, 256), 256, 0, ctx->stream>>>(x, len, R, s->maxbits, s->xs, s->e);
    ctx->launches += 2;
    e = cudaGetLastError();
    return e == cudaSuccess ? BEM_OK : ctx->fail(BEM_ERR_CUDA, std::string("df split: ") + cudaGetErrorString(e));
}

}  // namespace

// Complex128 matrix (n entries, device) -> scaled split form in place; the
// exponent is written to the device int *e.
int df_prepare_inplace(bem_ctx* ctx, double2* v, int64_t n, int* e) {
    DfScratch s;
    int rc = df_scratch(ctx, 1, 0, &s);
    if (rc) return rc;
    cudaError_t err = cudaMemsetAsync(s.maxbits, 0, sizeof(unsigned long long), ctx->stream);
    if (err != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string("df prepare: ") + cudaGetErrorString(err));
    df_maxbits_kernel<<<grid_for(n, 256), 256, 0, ctx->stream>>>(v, n, n, s.maxbits);
    df_split_inplace_kernel<<<grid_for(n, 256), 256, 0, ctx->stream>>>(v, n, s.maxbits, e);
    ctx->launches += 2;
    err = cudaGetLastError();
    return err == cudaSuccess ? BEM_OK : ctx->fail(BEM_ERR_CUDA, std::string("df prepare: ") + cudaGetErrorString(err));
}

// Y[r][i] = sum_j A[i][j] X[r][j] for r < R, A split (m x k, row stride lda).
int df_gemv(bem_ctx* ctx, const float4* A, const int* eA, int64_t m, int64_t k, int64_t lda, const double2* X,
            int64_t R, double2* Y, int64_t ldy) {
    DfScratch s;
    int rc = split_vectors(ctx, X, R, k, &s);
    if (rc) return rc;
    DfGemvArgs a{A, m, k, lda, eA, s.xs, s.e, R, Y, ldy};
    const int threads = DF_WARPS * 32;
    auto grid = [&](int rw) {
        const int64_t groups = (m + rw - 1) / rw;
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>((groups + DF_WARPS - 1) / DF_WARPS, 152 * 4));
    };
    if (R == 1) df_gemv_kernel<4, 1><<<grid(4), threads, 0, ctx->stream>>>(a);
    else if (R == 2) df_gemv_kernel<2, 2><<<grid(2), threads, 0, ctx->stream>>>(a);
    else df_gemv_kernel<2, 4><<<grid(2), threads, 0, ctx->stream>>>(a);  // (one row x 8 vectors per warp measured slower)
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BEM_OK : ctx->fail(BEM_ERR_CUDA, std::string("df gemv: ") + cudaGetErrorString(e));
}

// U[r][j] = sum_m W[r][m] B[m][j], B split (K x n), W complex128 [R][K].
int df_combine(bem_ctx* ctx, const float4* B, const int* eB, int64_t K, int64_t n, const double2* W, int64_t R,
               double2* U) {
    DfScratch s;
    int rc = split_vectors(ctx, W, R, K, &s);
    if (rc) return rc;
    DfCombineArgs a{B, K, n, eB, s.xs, s.e, R, U};
    constexpr int RG = 4;
    const dim3 grid((unsigned)((n + 255) / 256), (unsigned)((R + RG - 1) / RG));
    df_combine_kernel<RG><<<grid, 256, 0, ctx->stream>>>(a);
    ctx->launches += 1;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BEM_OK : ctx->fail(BEM_ERR_CUDA, std::string("df combine: ") + cudaGetErrorString(e));
}

}  // namespace gbem
