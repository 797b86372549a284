// k_krylov.cu -- restarted GMRES with FP64 device vectors (the paper's
// solver: GMRES, restart 100, Sec. 3).  Arnoldi by classical Gram-Schmidt
// applied twice (one batched dot-product kernel and one batched update per
// pass), deterministic fixed-order reductions.  The Hessenberg columns, the
// Givens rotations, the residual estimates and the triangular solve of each
// restart cycle stay on the device in FP64 (one small kernel per step), so an
// Arnoldi step does not wait for the host: the host reads how many columns
// are still running a few steps late (POLL_LAG) and stops launching steps
// once none is.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <functional>
#include <type_traits>
#include <vector>

#include "ctx.h"
#include "internal.h"
#include "krylov.h"

namespace gbem {

constexpr int KV_THREADS = 256;
constexpr int KV_BLOCKS = 120;

// part[k][blk] = sum_{i in blk} conj(V_k[i]) w[i]
__global__ void kv_dots(const double2* V, int64_t ldv, int nk, const double2* w, int64_t n, double2* part) {
    const int k = blockIdx.y;
    const double2* v = V + (int64_t)k * ldv;
    double sr = 0, si = 0;
    for (int64_t i = (int64_t)blockIdx.x * KV_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * KV_THREADS) {
        const double2 a = v[i], b = w[i];
        sr += a.x * b.x + a.y * b.y;
        si += a.x * b.y - a.y * b.x;
    }
    __shared__ double sh[2][KV_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = sr;
        sh[1][threadIdx.x >> 5] = si;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int q = 0; q < KV_THREADS / 32; q++) {
            a += sh[0][q];
            b += sh[1][q];
        }
        part[(int64_t)k * gridDim.x + blockIdx.x] = make_double2(a, b);
    }
}

// h[k] (+)= sum_blk part[k][blk]  (one block per k, fixed order)
__global__ void kv_reduce(const double2* part, int nblk, double2* h, int accumulate) {
    const int k = blockIdx.x;
    if (threadIdx.x != 0) return;
    double a = 0, b = 0;
    for (int q = 0; q < nblk; q++) {
        a += part[(int64_t)k * nblk + q].x;
        b += part[(int64_t)k * nblk + q].y;
    }
    if (accumulate) {
        h[k].x += a;
        h[k].y += b;
    } else {
        h[k] = make_double2(a, b);
    }
}

// w[i] -= sum_k c[k] V_k[i]   (c read from device)
__global__ void kv_subtract(const double2* V, int64_t ldv, int nk, const double2* c, double2* w, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * KV_THREADS + threadIdx.x;
    if (i >= n) return;
    double2 acc = w[i];
    for (int k = 0; k < nk; k++) {
        const double2 ck = c[k], v = V[(int64_t)k * ldv + i];
        acc.x -= ck.x * v.x - ck.y * v.y;
        acc.y -= ck.x * v.y + ck.y * v.x;
    }
    w[i] = acc;
}

// x[i] += sum_k y[k] V_k[i]
__global__ void kv_combine(const double2* V, int64_t ldv, int nk, const double2* y, double2* x, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * KV_THREADS + threadIdx.x;
    if (i >= n) return;
    double2 acc = x[i];
    for (int k = 0; k < nk; k++) {
        const double2 c = y[k], v = V[(int64_t)k * ldv + i];
        acc.x += c.x * v.x - c.y * v.y;
        acc.y += c.x * v.y + c.y * v.x;
    }
    x[i] = acc;
}

// y = a x (+ b z)
__global__ void kv_axpby(int64_t n, double2 a, const double2* x, double2 b, const double2* z, double2* y) {
    const int64_t i = (int64_t)blockIdx.x * KV_THREADS + threadIdx.x;
    if (i >= n) return;
    const double2 xi = x[i];
    double2 r = make_double2(a.x * xi.x - a.y * xi.y, a.x * xi.y + a.y * xi.x);
    if (z) {
        const double2 zi = z[i];
        r.x += b.x * zi.x - b.y * zi.y;
        r.y += b.x * zi.y + b.y * zi.x;
    }
    y[i] = r;
}

// ---- batched (R columns): a basis block k holds R columns of n, column r at k*ldk + r*n

// part[(r*nk + k)*nbk + blk] = sum_{i in blk} conj(V_{k,r}[i]) W_r[i]
__global__ void kvb_dots(const double2* V, int64_t ldk, int nk, const double2* W, int64_t n, int nbk, double2* part) {
    const int blk = blockIdx.x, k = blockIdx.y, r = blockIdx.z;
    const double2* v = V + (int64_t)k * ldk + (int64_t)r * n;
    const double2* w = W + (int64_t)r * n;
    double sr = 0, si = 0;
    for (int64_t i = (int64_t)blk * KV_THREADS + threadIdx.x; i < n; i += (int64_t)nbk * KV_THREADS) {
        const double2 a = v[i], b = w[i];
        sr += a.x * b.x + a.y * b.y;
        si += a.x * b.y - a.y * b.x;
    }
    __shared__ double sh[2][KV_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = sr;
        sh[1][threadIdx.x >> 5] = si;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int q = 0; q < KV_THREADS / 32; q++) {
            a += sh[0][q];
            b += sh[1][q];
        }
        part[((int64_t)r * nk + k) * nbk + blk] = make_double2(a, b);
    }
}

// h[r*ldh + k] = sum_blk part[(r*nk + k)*nbk + blk]   (grid nk x R, fixed order)
__global__ void kvb_reduce(const double2* part, int nk, int nbk, double2* h, int ldh) {
    const int k = blockIdx.x, r = blockIdx.y;
    if (threadIdx.x != 0) return;
    double a = 0, b = 0;
    const double2* p = part + ((int64_t)r * nk + k) * nbk;
    for (int q = 0; q < nbk; q++) {
        a += p[q].x;
        b += p[q].y;
    }
    h[(int64_t)r * ldh + k] = make_double2(a, b);
}

// W_r[i] -= sum_k c[r*ldh + k] V_{k,r}[i]    (sign = -1), or X_r += ... (sign = +1)
__global__ void kvb_update(const double2* V, int64_t ldk, int nk, const double2* c, int ldh, double2* W, int64_t n,
                           double sign) {
    const int64_t i = (int64_t)blockIdx.x * KV_THREADS + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= n) return;
    double2 acc = W[(int64_t)r * n + i];
    const double2* cr = c + (int64_t)r * ldh;
    for (int k = 0; k < nk; k++) {
        const double2 ck = cr[k], v = V[(int64_t)k * ldk + (int64_t)r * n + i];
        acc.x += sign * (ck.x * v.x - ck.y * v.y);
        acc.y += sign * (ck.x * v.y + ck.y * v.x);
    }
    W[(int64_t)r * n + i] = acc;
}

// W_r *= s[r]
__global__ void kvb_scale(double2* W, int64_t n, const double* s) {
    const int64_t i = (int64_t)blockIdx.x * KV_THREADS + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= n) return;
    double2 v = W[(int64_t)r * n + i];
    v.x *= s[r];
    v.y *= s[r];
    W[(int64_t)r * n + i] = v;
}

// ---- block GMRES: products between a basis of K vectors and P columns

constexpr int KB_COLS = 16;  // columns handled per pass of the block kernels

// part[(k P + c) nsplit + blk] = sum_{i in blk} conj(V_k[i]) W_c[i] for the
// KB_COLS columns c0 .. c0 + KB_COLS - 1 (those below P); grid (K, nsplit).
__global__ void __launch_bounds__(KV_THREADS) kbd_dots(int64_t n, int K, int P, const double2* __restrict__ V,
                                                       const double2* __restrict__ W, int c0, int nsplit,
                                                       double2* __restrict__ part) {
    const int k = blockIdx.x, blk = blockIdx.y;
    const int nc = min(KB_COLS, P - c0);
    double ar[KB_COLS], ai[KB_COLS];
#pragma unroll
    for (int c = 0; c < KB_COLS; c++) ar[c] = ai[c] = 0.0;
    const double2* v = V + (int64_t)k * n;
    for (int64_t i = (int64_t)blk * KV_THREADS + threadIdx.x; i < n; i += (int64_t)nsplit * KV_THREADS) {
        const double2 a = v[i];
#pragma unroll
        for (int c = 0; c < KB_COLS; c++)
            if (c < nc) {
                const double2 b = W[(int64_t)(c0 + c) * n + i];
                ar[c] += a.x * b.x + a.y * b.y;
                ai[c] += a.x * b.y - a.y * b.x;
            }
    }
    __shared__ double sh[KV_THREADS / 32][KB_COLS][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < KB_COLS; c++) {
        double x = ar[c], y = ai[c];
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if (lane == 0) {
            sh[warp][c][0] = x;
            sh[warp][c][1] = y;
        }
    }
    __syncthreads();
    if (threadIdx.x < nc) {
        double x = 0, y = 0;
        for (int w = 0; w < KV_THREADS / 32; w++) {
            x += sh[w][threadIdx.x][0];
            y += sh[w][threadIdx.x][1];
        }
        part[((int64_t)k * P + c0 + threadIdx.x) * nsplit + blk] = make_double2(x, y);
    }
}

// C[k P + c] = sum_blk part[(k P + c) nsplit + blk]  (fixed order)
// Back substitution Y = R^-1 G of the block GMRES least squares, by blocks of
// BS_ROWS rows from the bottom: R upper triangular J x J (column-major,
// leading dimension ld), G [J][P] row-major (overwritten), Y [J][P]; a zero
// pivot gives a zero row of Y.  bs_block_kernel (one CTA, thread (r, c))
// solves rows [i0, i1) against the block's own columns; bs_update_kernel
// (thread per (row, column) above i0) subtracts those columns' part.
constexpr int BS_ROWS = 32;
__device__ __forceinline__ double2 cdiv(double2 g, double2 d) {
    const double dd = d.x * d.x + d.y * d.y;
    return dd > 0 ? make_double2((g.x * d.x + g.y * d.y) / dd, (g.y * d.x - g.x * d.y) / dd) : make_double2(0, 0);
}
__global__ void bs_block_kernel(const double2* __restrict__ R, int64_t ld, double2* __restrict__ G,
                                double2* __restrict__ Y, int P, int i0, int i1) {
    __shared__ double2 ys[32];
    const int c = threadIdx.x, r = threadIdx.y;  // blockDim = (P, BS_ROWS)
    for (int i = i1 - 1; i >= i0; i--) {
        if (r == i - i0) {
            const double2 y = cdiv(G[(int64_t)i * P + c], R[(int64_t)i * ld + i]);
            Y[(int64_t)i * P + c] = y;
            ys[c] = y;
        }
        __syncthreads();
        if (r < i - i0) {
            const double2 h = R[(int64_t)i * ld + i0 + r], y = ys[c];
            double2& g = G[(int64_t)(i0 + r) * P + c];
            g.x -= h.x * y.x - h.y * y.y;
            g.y -= h.x * y.y + h.y * y.x;
        }
        __syncthreads();
    }
}
__global__ void bs_update_kernel(const double2* __restrict__ R, int64_t ld, double2* __restrict__ G,
                                 const double2* __restrict__ Y, int P, int i0, int i1) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = t / P;
    const int c = (int)(t % P);
    if (r >= i0) return;
    double sr = 0, si = 0;
    for (int i = i0; i < i1; i++) {
        const double2 h = R[(int64_t)i * ld + r], y = Y[(int64_t)i * P + c];
        sr += h.x * y.x - h.y * y.y;
        si += h.x * y.y + h.y * y.x;
    }
    double2& g = G[r * P + c];
    g.x -= sr;
    g.y -= si;
}

__global__ void kbd_reduce(int KP, int nsplit, const double2* __restrict__ part, double2* __restrict__ C) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= KP) return;
    double x = 0, y = 0;
    for (int q = 0; q < nsplit; q++) {
        x += part[(int64_t)e * nsplit + q].x;
        y += part[(int64_t)e * nsplit + q].y;
    }
    C[e] = make_double2(x, y);
}

// out_c[i] = beta base_c[i] + alpha sum_k V_k[i] C[k P + c] for the columns
// c0 .. c0 + KB_COLS - 1 below P (base may be null; out may equal base, not V).
__global__ void __launch_bounds__(KV_THREADS) kbd_combine(int64_t n, int K, int P, const double2* __restrict__ V,
                                                          const double2* __restrict__ C, double alpha,
                                                          const double2* base, double beta, double2* out, int c0) {
    __shared__ double2 cs[64][KB_COLS];
    const int64_t i = (int64_t)blockIdx.x * KV_THREADS + threadIdx.x;
    const int nc = min(KB_COLS, P - c0);
    double ar[KB_COLS], ai[KB_COLS];
#pragma unroll
    for (int c = 0; c < KB_COLS; c++) {
        ar[c] = ai[c] = 0.0;
        if (base && c < nc && i < n) {
            const double2 b = base[(int64_t)(c0 + c) * n + i];
            ar[c] = beta * b.x;
            ai[c] = beta * b.y;
        }
    }
    for (int k0 = 0; k0 < K; k0 += 64) {
        const int kn = min(64, K - k0);
        __syncthreads();
        for (int e = threadIdx.x; e < kn * KB_COLS; e += KV_THREADS) {
            const int kk = e / KB_COLS, c = e % KB_COLS;
            const double2 v = c < nc ? C[(int64_t)(k0 + kk) * P + c0 + c] : make_double2(0, 0);
            cs[kk][c] = make_double2(alpha * v.x, alpha * v.y);
        }
        __syncthreads();
        if (i < n)
            for (int kk = 0; kk < kn; kk++) {
                const double2 v = V[(int64_t)(k0 + kk) * n + i];
#pragma unroll
                for (int c = 0; c < KB_COLS; c++) {
                    const double2 cc = cs[kk][c];
                    ar[c] += v.x * cc.x - v.y * cc.y;
                    ai[c] += v.x * cc.y + v.y * cc.x;
                }
            }
    }
    if (i < n)
#pragma unroll
        for (int c = 0; c < KB_COLS; c++)
            if (c < nc) out[(int64_t)(c0 + c) * n + i] = make_double2(ar[c], ai[c]);
}

// FP32 forms of the two block kernels (the inner solves of the mixed path,
// whose tolerance (1e-4) needs no FP64 orthogonalisation): FP32 vectors and
// arithmetic, per-block partial sums returned in FP64.
// FP32 block dots as a tiled contraction: CTA (x, y) forms the 64 x KB_COLS
// tile of C = V^H W for rows 64 x .. 64 x + 63 and the columns c0 .. over the
// y-th slice of n, staging 32 entries of each row and column in shared memory
// per step (V read once from memory, W once per row tile).  Thread (ty, tx)
// accumulates rows ty + 16 r (r < 4) of column tx; each 32-entry chunk is
// summed in FP32 and folded into a compensated (Kahan) FP32 total, which is
// written as FP64 partials part[(k P + c) nsplit + y].
constexpr int KD_ROWS = 64, KD_CHUNK = 32;
__global__ void __launch_bounds__(KV_THREADS) kbd_dots32(int64_t n, int K, int P, const float2* __restrict__ V,
                                                         const float2* __restrict__ W, int c0, int nsplit,
                                                         int64_t slice, double2* __restrict__ part) {
    __shared__ float2 vs[KD_ROWS][KD_CHUNK + 1];
    __shared__ float2 ws[KB_COLS][KD_CHUNK + 1];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int k0 = blockIdx.x * KD_ROWS, blk = blockIdx.y;
    const int nc = min(KB_COLS, P - c0);
    const int64_t i_begin = (int64_t)blk * slice, i_end = min(n, i_begin + slice);
    float tr[4], ti[4], cr[4], ci[4];
#pragma unroll
    for (int r = 0; r < 4; r++) tr[r] = ti[r] = cr[r] = ci[r] = 0.f;
    for (int64_t i0 = i_begin; i0 < i_end; i0 += KD_CHUNK) {
#pragma unroll
        for (int l = 0; l < KD_ROWS * KD_CHUNK / KV_THREADS; l++) {
            const int idx = l * KV_THREADS + t, row = idx / KD_CHUNK, e = idx % KD_CHUNK;
            const int64_t i = i0 + e;
            vs[row][e] = (k0 + row < K && i < i_end) ? V[(int64_t)(k0 + row) * n + i] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int l = 0; l < KB_COLS * KD_CHUNK / KV_THREADS; l++) {
            const int idx = l * KV_THREADS + t, col = idx / KD_CHUNK, e = idx % KD_CHUNK;
            const int64_t i = i0 + e;
            ws[col][e] = (col < nc && i < i_end) ? W[(int64_t)(c0 + col) * n + i] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
        for (int e = 0; e < KD_CHUNK; e++) {
            const float2 b = ws[tx][e];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const float2 a = vs[ty + 16 * r][e];
                ar[r] = fmaf(a.x, b.x, fmaf(a.y, b.y, ar[r]));
                ai[r] = fmaf(a.x, b.y, fmaf(-a.y, b.x, ai[r]));
            }
        }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            float y = ar[r] - cr[r], u = tr[r] + y;
            cr[r] = (u - tr[r]) - y;
            tr[r] = u;
            y = ai[r] - ci[r];
            u = ti[r] + y;
            ci[r] = (u - ti[r]) - y;
            ti[r] = u;
        }
        __syncthreads();
    }
    if (tx >= nc) return;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int k = k0 + ty + 16 * r;
        if (k < K)
            part[((int64_t)k * P + c0 + tx) * nsplit + blk] =
                make_double2((double)tr[r] - (double)cr[r], (double)ti[r] - (double)ci[r]);
    }
}

__global__ void __launch_bounds__(KV_THREADS) kbd_combine32(int64_t n, int K, int P, const float2* __restrict__ V,
                                                            const double2* __restrict__ C, float alpha,
                                                            const float2* base, float beta, float2* out, int c0) {
    __shared__ float2 cs[64][KB_COLS];
    const int64_t i = (int64_t)blockIdx.x * KV_THREADS + threadIdx.x;
    const int nc = min(KB_COLS, P - c0);
    float ar[KB_COLS], ai[KB_COLS];
#pragma unroll
    for (int c = 0; c < KB_COLS; c++) {
        ar[c] = ai[c] = 0.f;
        if (base && c < nc && i < n) {
            const float2 b = base[(int64_t)(c0 + c) * n + i];
            ar[c] = beta * b.x;
            ai[c] = beta * b.y;
        }
    }
    for (int k0 = 0; k0 < K; k0 += 64) {
        const int kn = min(64, K - k0);
        __syncthreads();
        for (int e = threadIdx.x; e < kn * KB_COLS; e += KV_THREADS) {
            const int kk = e / KB_COLS, c = e % KB_COLS;
            const double2 v = c < nc ? C[(int64_t)(k0 + kk) * P + c0 + c] : make_double2(0, 0);
            cs[kk][c] = make_float2(alpha * (float)v.x, alpha * (float)v.y);
        }
        __syncthreads();
        if (i < n)
#pragma unroll 4
            for (int kk = 0; kk < kn; kk++) {
                const float2 v = V[(int64_t)(k0 + kk) * n + i];
#pragma unroll
                for (int c = 0; c < KB_COLS; c++) {
                    const float2 cc = cs[kk][c];
                    ar[c] = fmaf(v.x, cc.x, fmaf(-v.y, cc.y, ar[c]));
                    ai[c] = fmaf(v.x, cc.y, fmaf(v.y, cc.x, ai[c]));
                }
            }
    }
    if (i < n)
#pragma unroll
        for (int c = 0; c < KB_COLS; c++)
            if (c < nc) out[(int64_t)(c0 + c) * n + i] = make_float2(ar[c], ai[c]);
}

__global__ void kv_to32(int64_t len, const double2* __restrict__ a, float2* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * KV_THREADS + threadIdx.x;
    if (i < len) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void kv_to64(int64_t len, const float2* __restrict__ a, double2* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * KV_THREADS + threadIdx.x;
    if (i < len) b[i] = make_double2((double)a[i].x, (double)a[i].y);
}

// ---- least squares on the device

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

struct GivensArgs {
    const double2* part;   // [R][nbk] partial sums of |v_{j+1}|^2 (real parts)
    int nbk;
    const double2* h1;     // [R][ldh] first Gram-Schmidt pass
    const double2* h2;     // [R][ldh] second pass
    int ldh, j, m;
    double2 *H, *cs, *sn, *g;
    const double* bn;
    double* res;
    int *run, *jr, *its;
    double* scale;         // [R] 1 / h_{j+1,j} for running columns, else 0
    double tol;
    int* n_run;            // running columns after this step (zeroed before the launch)
};

// Step j of every column: Hessenberg column j = h1 + h2 and |v_{j+1}|, the
// earlier rotations applied to it, the new rotation that zeroes h_{j+1,j},
// the rotated right-hand side g and the residual estimate |g_{j+1}| / |b|.
__global__ void givens_step_kernel(GivensArgs a) {
    const int r = blockIdx.x;
    if (threadIdx.x != 0) return;
    a.scale[r] = 0.0;
    if (!a.run[r]) return;
    const int m = a.m, j = a.j;
    double s = 0;
    for (int q = 0; q < a.nbk; q++) s += a.part[(int64_t)r * a.nbk + q].x;
    const double hn = sqrt(fmax(0.0, s));
    double2* H = a.H + (int64_t)r * (m + 1) * m;
    double2* cs = a.cs + (int64_t)r * m;
    double2* sn = a.sn + (int64_t)r * m;
    double2* g = a.g + (int64_t)r * (m + 1);
    for (int i = 0; i <= j; i++) H[i * m + j] = zadd(a.h1[(int64_t)r * a.ldh + i], a.h2[(int64_t)r * a.ldh + i]);
    H[(j + 1) * m + j] = make_double2(hn, 0.0);
    for (int i = 0; i < j; i++) {
        const double2 x = H[i * m + j], y = H[(i + 1) * m + j];
        H[i * m + j] = zadd(zmul(zconj(cs[i]), x), zmul(zconj(sn[i]), y));
        H[(i + 1) * m + j] = zsub(zmul(cs[i], y), zmul(sn[i], x));
    }
    const double2 x = H[j * m + j], y = H[(j + 1) * m + j];
    const double den = sqrt(x.x * x.x + x.y * x.y + y.x * y.x + y.y * y.y);
    cs[j] = den > 0 ? make_double2(x.x / den, x.y / den) : make_double2(1.0, 0.0);
    sn[j] = den > 0 ? make_double2(y.x / den, y.y / den) : make_double2(0.0, 0.0);
    H[j * m + j] = make_double2(den, 0.0);
    H[(j + 1) * m + j] = make_double2(0.0, 0.0);
    const double2 gj = g[j];
    g[j + 1] = zmul(make_double2(-sn[j].x, -sn[j].y), gj);
    g[j] = zmul(zconj(cs[j]), gj);
    a.its[r] += 1;
    a.jr[r] = j + 1;
    const double rr = sqrt(g[j + 1].x * g[j + 1].x + g[j + 1].y * g[j + 1].y) / a.bn[r];
    a.res[r] = rr;
    if (rr <= a.tol || hn == 0) {
        a.run[r] = 0;
    } else {
        a.scale[r] = 1.0 / hn;
        atomicAdd(a.n_run, 1);
    }
}

// y = H^-1 g over each column's own jr steps (zeros beyond), FP64.
__global__ void backsolve_kernel(const double2* H, const double2* g, const int* jr, int m, double2* y, int ldh) {
    const int r = blockIdx.x;
    if (threadIdx.x != 0) return;
    const double2* Hr = H + (int64_t)r * (m + 1) * m;
    const double2* gr = g + (int64_t)r * (m + 1);
    double2* yr = y + (int64_t)r * ldh;
    const int jj = jr[r];
    for (int i = jj; i < ldh; i++) yr[i] = make_double2(0.0, 0.0);
    for (int i = jj - 1; i >= 0; i--) {
        double2 s = gr[i];
        for (int k = i + 1; k < jj; k++) s = zsub(s, zmul(Hr[i * m + k], yr[k]));
        yr[i] = zdiv(s, Hr[i * m + i]);
    }
}

}  // namespace gbem

using namespace gbem;

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int Krylov::ensure(bem_ctx* ctx, int64_t n_, int m_, int64_t R_) {
    if (n == n_ && m >= m_ && R >= R_) return BEM_OK;
    const int mm = std::max(m_, n == n_ ? m : 0);
    const int64_t RR = std::max<int64_t>(R_, n == n_ ? R : 1);
    release(ctx);
    n = n_;
    m = mm;
    R = RR;
    int rc;
    V = (double2*)ctx->dalloc((size_t)(m + 1) * R * n * sizeof(double2), &rc); if (rc) return rc;
    w = (double2*)ctx->dalloc(R * n * sizeof(double2), &rc); if (rc) return rc;
    t = (double2*)ctx->dalloc(R * n * sizeof(double2), &rc); if (rc) return rc;
    part = (double2*)ctx->dalloc((size_t)(m + 2) * KV_BLOCKS * R * sizeof(double2), &rc); if (rc) return rc;
    h = (double2*)ctx->dalloc((m + 2) * R * sizeof(double2), &rc); if (rc) return rc;
    y = (double2*)ctx->dalloc((m + 2) * R * sizeof(double2), &rc); if (rc) return rc;
    sc = (double*)ctx->dalloc(R * sizeof(double), &rc); if (rc) return rc;
    H = (double2*)ctx->dalloc((size_t)R * (m + 1) * m * sizeof(double2), &rc); if (rc) return rc;
    cs = (double2*)ctx->dalloc((size_t)R * m * sizeof(double2), &rc); if (rc) return rc;
    sn = (double2*)ctx->dalloc((size_t)R * m * sizeof(double2), &rc); if (rc) return rc;
    g = (double2*)ctx->dalloc((size_t)R * (m + 1) * sizeof(double2), &rc); if (rc) return rc;
    bn = (double*)ctx->dalloc(R * sizeof(double), &rc); if (rc) return rc;
    res = (double*)ctx->dalloc(R * sizeof(double), &rc); if (rc) return rc;
    run = (int*)ctx->dalloc(R * sizeof(int), &rc); if (rc) return rc;
    jr = (int*)ctx->dalloc(R * sizeof(int), &rc); if (rc) return rc;
    its = (int*)ctx->dalloc(R * sizeof(int), &rc); if (rc) return rc;
    n_run = (int*)ctx->dalloc(4 * sizeof(int), &rc); if (rc) return rc;
    if (!n_run_host && cudaMallocHost(&n_run_host, 4 * sizeof(int)) != cudaSuccess) {
        n_run_host = nullptr;
        return ctx->fail(BEM_ERR_CUDA, "cudaMallocHost (GMRES poll)");
    }
    for (auto& e : poll_ev)
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return ctx->fail(BEM_ERR_CUDA, "cudaEventCreate (GMRES poll)");
    return BEM_OK;
}

void Krylov::dfree_buf(bem_ctx* ctx, void** p) {
    ctx->dfree(*p);
    *p = nullptr;
}

int Krylov::ensure_flexible(bem_ctx* ctx) {
    if (Z) return BEM_OK;
    int rc;
    Z = (double2*)ctx->dalloc((size_t)m * R * n * sizeof(double2), &rc);
    return rc;
}

void Krylov::release(bem_ctx* ctx) {
    for (void* p : {(void*)V, (void*)w, (void*)t, (void*)part, (void*)h, (void*)y, (void*)sc, (void*)Z, (void*)H,
                    (void*)cs, (void*)sn, (void*)g, (void*)bn, (void*)res, (void*)run, (void*)jr, (void*)its,
                    (void*)n_run, (void*)bpart, (void*)bC, (void*)b32})
        ctx->dfree(p);
    V = w = t = part = h = y = Z = H = cs = sn = g = bpart = bC = nullptr;
    b32 = nullptr;
    bpart_n = bC_n = b32_n = 0;
    sc = bn = res = nullptr;
    run = jr = its = n_run = nullptr;
    n = 0;
    m = 0;
    R = 0;
}

int Krylov::dot(bem_ctx* ctx, const double2* a, const double2* b, std::complex<double>* out) {
    // reduce into the last slot of h (never used by an Arnoldi column)
    kv_dots<<<dim3(KV_BLOCKS, 1), KV_THREADS, 0, ctx->stream>>>(a, n, 1, b, n, part);
    kv_reduce<<<1, 32, 0, ctx->stream>>>(part, KV_BLOCKS, h + m + 1, 0);
    double2 r;
    CK(cudaMemcpyAsync(&r, h + m + 1, sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->launches += 2;
    *out = {r.x, r.y};
    return BEM_OK;
}

int Krylov::norm(bem_ctx* ctx, const double2* a, double* out) {
    std::complex<double> d;
    int rc = dot(ctx, a, a, &d);
    *out = std::sqrt(std::max(0.0, d.real()));
    return rc;
}

int Krylov::axpby(bem_ctx* ctx, std::complex<double> a, const double2* x, std::complex<double> b, const double2* z,
                  double2* out, int64_t len) {
    if (len < 0) len = n;
    const unsigned nb = (unsigned)((len + KV_THREADS - 1) / KV_THREADS);
    kv_axpby<<<nb, KV_THREADS, 0, ctx->stream>>>(len, make_double2(a.real(), a.imag()), x,
                                                 make_double2(b.real(), b.imag()), z, out);
    ctx->launches += 1;
    CK(cudaGetLastError());
    return BEM_OK;
}

// Solve op(x) = b to ||b - op(x)|| <= tol ||b|| (residual of the system it is
// given), x holds the initial guess on entry: the batched solver with one column.
int Krylov::gmres(bem_ctx* ctx, const Op& op, const double2* b, double2* x, int restart, double tol, int max_iter,
                  int* iters, double* relres, bool zero_guess, const Op* prec) {
    return gmres_batch(ctx, op, b, x, 1, restart, tol, max_iter, iters, relres, zero_guess, prec);
}

// ---------------------------------------------------------------- batched GMRES

// blocks per (column, basis vector) of a batched dot: enough CTAs in total to
// fill the GPU, at most KV_BLOCKS, at most what n needs
static int batch_blocks(int64_t n, int64_t cols) {
    const int64_t need = (n + KV_THREADS - 1) / KV_THREADS;
    const int64_t want = (4 * 152 + cols - 1) / cols;
    return (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)KV_BLOCKS, need, want}));
}

int Krylov::norms(bem_ctx* ctx, const double2* a, int64_t Rn, double* out) {
    const int nbk = batch_blocks(n, Rn);
    kvb_dots<<<dim3(nbk, 1, (unsigned)Rn), KV_THREADS, 0, ctx->stream>>>(a, 0, 1, a, n, nbk, part);
    kvb_reduce<<<dim3(1, (unsigned)Rn), 32, 0, ctx->stream>>>(part, 1, nbk, h, 1);
    ctx->launches += 2;
    std::vector<double2> hv(Rn);
    CK(cudaMemcpyAsync(hv.data(), h, Rn * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int64_t r = 0; r < Rn; r++) out[r] = std::sqrt(std::max(0.0, hv[r].x));
    return BEM_OK;
}

int Krylov::gmres_batch(bem_ctx* ctx, const Op& op, const double2* B, double2* X, int64_t Rn, int restart,
                        double tol, int max_iter, int* iters, double* relres, bool zero_guess, const Op* prec) {
    int rc = ensure(ctx, n, restart, Rn);
    if (rc) return rc;
    if (prec && (rc = ensure_flexible(ctx))) return rc;
    constexpr int POLL_LAG = 2;  // steps the host may run ahead of the last running-count it has seen
    const int64_t ldk = Rn * n;  // stride between basis blocks
    const int ldh = m + 2;
    const unsigned nb = (unsigned)((n + KV_THREADS - 1) / KV_THREADS);
    const dim3 gcol(nb, (unsigned)Rn);
    std::vector<double> bnorm(Rn), beta(Rn), scale(Rn), resv(Rn, 0.0);
    if ((rc = norms(ctx, B, Rn, bnorm.data()))) return rc;
    std::vector<char> live(Rn);
    for (int64_t r = 0; r < Rn; r++) {
        iters[r] = 0;
        live[r] = bnorm[r] > 0;
    }
    CK(cudaMemcpyAsync(bn, bnorm.data(), Rn * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(its, 0, Rn * sizeof(int), ctx->stream));
    std::vector<double2> g0((size_t)(m + 1) * Rn);
    std::vector<int> run0(Rn), itv(Rn);
    int total = 0;
    bool first = true;
    while (total < max_iter) {
        // residual block into V_0
        if (first && zero_guess) {
            CK(cudaMemcpyAsync(V, B, Rn * n * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaMemsetAsync(X, 0, Rn * n * sizeof(double2), ctx->stream));
        } else {
            if ((rc = op(X, t))) return rc;
            kv_axpby<<<(unsigned)((Rn * n + KV_THREADS - 1) / KV_THREADS), KV_THREADS, 0, ctx->stream>>>(
                Rn * n, make_double2(1, 0), B, make_double2(-1, 0), t, V);
            ctx->launches += 1;
        }
        first = false;
        if ((rc = norms(ctx, V, Rn, beta.data()))) return rc;  // synchronises (once per restart cycle)
        bool any = false;
        std::fill(g0.begin(), g0.end(), make_double2(0, 0));
        for (int64_t r = 0; r < Rn; r++) {
            if (live[r]) resv[r] = beta[r] / bnorm[r];
            const bool go = live[r] && resv[r] > tol;
            live[r] = go;
            any |= go;
            run0[r] = go;
            scale[r] = go ? 1.0 / beta[r] : 0.0;  // finished columns carry zeros
            g0[(size_t)r * (m + 1)] = make_double2(go ? beta[r] : 0.0, 0.0);
        }
        if (!any) break;
        CK(cudaMemcpyAsync(sc, scale.data(), Rn * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(g, g0.data(), g0.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(run, run0.data(), Rn * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemsetAsync(jr, 0, Rn * sizeof(int), ctx->stream));
        kvb_scale<<<gcol, KV_THREADS, 0, ctx->stream>>>(V, n, sc);
        ctx->launches += 1;
        int j = 0, polled = 0;
        for (; j < restart && total < max_iter; j++) {
            double2* vj1 = V + (int64_t)(j + 1) * ldk;
            if (prec) {
                double2* zj = Z + (int64_t)j * ldk;
                if ((rc = (*prec)(V + (int64_t)j * ldk, zj))) return rc;
                if ((rc = op(zj, vj1))) return rc;
            } else if ((rc = op(V + (int64_t)j * ldk, vj1))) {
                return rc;
            }
            const int nbk = batch_blocks(n, Rn * (j + 1));
            for (int pass = 0; pass < 2; pass++) {
                double2* hp = pass == 0 ? h : y;
                kvb_dots<<<dim3(nbk, j + 1, (unsigned)Rn), KV_THREADS, 0, ctx->stream>>>(V, ldk, j + 1, vj1, n, nbk, part);
                kvb_reduce<<<dim3(j + 1, (unsigned)Rn), 32, 0, ctx->stream>>>(part, j + 1, nbk, hp, ldh);
                kvb_update<<<gcol, KV_THREADS, 0, ctx->stream>>>(V, ldk, j + 1, hp, ldh, vj1, n, -1.0);
                ctx->launches += 3;
            }
            // |v_{j+1}|^2 partials, then the least-squares step of every column
            const int nb1 = batch_blocks(n, Rn);
            kvb_dots<<<dim3(nb1, 1, (unsigned)Rn), KV_THREADS, 0, ctx->stream>>>(vj1, 0, 1, vj1, n, nb1, part);
            const int slot = j % 4;
            CK(cudaMemsetAsync(n_run + slot, 0, sizeof(int), ctx->stream));
            GivensArgs ga{part, nb1, h, y, ldh, j, m, H, cs, sn, g, bn, res, run, jr, its, sc, tol, n_run + slot};
            givens_step_kernel<<<(unsigned)Rn, 32, 0, ctx->stream>>>(ga);
            kvb_scale<<<gcol, KV_THREADS, 0, ctx->stream>>>(vj1, n, sc);
            CK(cudaMemcpyAsync(n_run_host + slot, n_run + slot, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaEventRecord(poll_ev[slot], ctx->stream));
            ctx->launches += 3;
            CK(cudaGetLastError());
            total++;
            // read the running counts of finished steps; wait only for the one POLL_LAG steps back
            bool done = false;
            while (polled <= j) {
                const cudaError_t q = polled <= j - POLL_LAG ? cudaEventSynchronize(poll_ev[polled % 4])
                                                             : cudaEventQuery(poll_ev[polled % 4]);
                if (q == cudaErrorNotReady) break;
                if (q != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string("GMRES poll: ") + cudaGetErrorString(q));
                if (n_run_host[polled % 4] == 0) {
                    done = true;
                    break;
                }
                polled++;
            }
            if (done) {
                j++;
                break;
            }
        }
        // back substitution per column (its own length) and X += V y
        backsolve_kernel<<<(unsigned)Rn, 32, 0, ctx->stream>>>(H, g, jr, m, y, ldh);
        ctx->launches += 1;
        if (j > 0) {
            kvb_update<<<gcol, KV_THREADS, 0, ctx->stream>>>(prec ? Z : V, ldk, j, y, ldh, X, n, 1.0);
            ctx->launches += 1;
        }
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(resv.data(), res, Rn * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(itv.data(), its, Rn * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        bool open = false;
        for (int64_t r = 0; r < Rn; r++) {
            iters[r] = itv[r];
            open |= live[r] && resv[r] > tol;
        }
        if (!open) break;
    }
    // true residuals of the given systems
    if ((rc = op(X, t))) return rc;
    kv_axpby<<<(unsigned)((Rn * n + KV_THREADS - 1) / KV_THREADS), KV_THREADS, 0, ctx->stream>>>(
        Rn * n, make_double2(1, 0), B, make_double2(-1, 0), t, t);
    ctx->launches += 1;
    std::vector<double> rn(Rn);
    if ((rc = norms(ctx, t, Rn, rn.data()))) return rc;
    for (int64_t r = 0; r < Rn; r++) relres[r] = bnorm[r] > 0 ? rn[r] / bnorm[r] : 0.0;
    return BEM_OK;
}

// ---------------------------------------------------------------- block GMRES

namespace {

using zd = std::complex<double>;

// slices of n for the tiled FP32 dots: about 4 x 152 CTAs in all, slices of
// at least 8 chunks; nsplit x gx <= max(gx, 608)
int nsplit_tiled(int64_t n, int gx) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 8 * KD_CHUNK - 1) / (8 * KD_CHUNK), 4 * 152 / gx));
}

int nsplit_for(int64_t n, int K) {
    return (int)std::max<int64_t>(1, std::min<int64_t>({8, (n + KV_THREADS - 1) / KV_THREADS,
                                                         (4 * 152 + K - 1) / std::max(1, K)}));
}

// C [K][P] (device, FP64) = V[0:K]^H W for P columns of n, FP64 or FP32 vectors.
template <class T>
int block_dots(bem_ctx* ctx, Krylov& k, const T* V, int K, const T* W, int P, double2* C) {
    const int64_t n = k.n;
    constexpr bool F32 = std::is_same<T, float2>::value;
    // FP32: row tiles of KD_ROWS, slices of whole chunks, about 4 CTAs per SM
    const int gx = F32 ? (K + KD_ROWS - 1) / KD_ROWS : K;
    const int nsplit = F32 ? nsplit_tiled(n, gx) : nsplit_for(n, K);
    const int64_t slice = F32 ? ((n + nsplit - 1) / nsplit + KD_CHUNK - 1) / KD_CHUNK * KD_CHUNK : 0;
    for (int c0 = 0; c0 < P; c0 += KB_COLS) {
        if constexpr (std::is_same<T, double2>::value)
            kbd_dots<<<dim3((unsigned)K, (unsigned)nsplit), KV_THREADS, 0, ctx->stream>>>(n, K, P, V, W, c0, nsplit,
                                                                                         k.bpart);
        else
            kbd_dots32<<<dim3((unsigned)gx, (unsigned)nsplit), KV_THREADS, 0, ctx->stream>>>(n, K, P, V, W, c0, nsplit,
                                                                                            slice, k.bpart);
    }
    kbd_reduce<<<(unsigned)((K * P + 127) / 128), 128, 0, ctx->stream>>>(K * P, nsplit, k.bpart, C);
    ctx->launches += (P + KB_COLS - 1) / KB_COLS + 1;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BEM_OK : ctx->fail(BEM_ERR_CUDA, std::string("block dots: ") + cudaGetErrorString(e));
}

// out = beta base + alpha V[0:K] C (C [K][P] device FP64), column groups of KB_COLS.
template <class T>
int block_combine(bem_ctx* ctx, int64_t n, const T* V, int K, int P, const double2* C, double alpha, const T* base,
                  double beta, T* out) {
    const unsigned nb = (unsigned)((n + KV_THREADS - 1) / KV_THREADS);
    for (int c0 = 0; c0 < P; c0 += KB_COLS) {
        if constexpr (std::is_same<T, double2>::value)
            kbd_combine<<<nb, KV_THREADS, 0, ctx->stream>>>(n, K, P, V, C, alpha, base, beta, out, c0);
        else
            kbd_combine32<<<nb, KV_THREADS, 0, ctx->stream>>>(n, K, P, V, C, (float)alpha, base, (float)beta, out, c0);
    }
    ctx->launches += (P + KB_COLS - 1) / KB_COLS;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BEM_OK : ctx->fail(BEM_ERR_CUDA, std::string("block combine: ") + cudaGetErrorString(e));
}

// In place: lower-triangular L with G = L L^H (G Hermitian P x P, row-major,
// unit diagonal up to rounding).  Returns false if a pivot falls to piv_min
// or below: the columns are dependent to within the vectors' precision.
bool cholesky(std::vector<zd>& G, int P, double piv_min) {
    for (int j = 0; j < P; j++) {
        double d = G[(size_t)j * P + j].real();
        for (int k2 = 0; k2 < j; k2++) d -= std::norm(G[(size_t)j * P + k2]);
        if (!(d > piv_min)) return false;
        const double l = std::sqrt(d);
        G[(size_t)j * P + j] = l;
        for (int i = j + 1; i < P; i++) {
            zd s = G[(size_t)i * P + j];
            for (int k2 = 0; k2 < j; k2++) s -= G[(size_t)i * P + k2] * std::conj(G[(size_t)j * P + k2]);
            G[(size_t)i * P + j] = s / l;
        }
        for (int i = 0; i < j; i++) G[(size_t)i * P + j] = 0.0;
    }
    return true;
}

// U^-1 for U = L^H (L lower triangular, row-major), row-major.
std::vector<zd> upper_inverse(const std::vector<zd>& L, int P) {
    std::vector<zd> Ui((size_t)P * P, zd(0));
    for (int c = 0; c < P; c++)
        for (int i = c; i >= 0; i--) {
            zd s = i == c ? 1.0 : 0.0;
            for (int k2 = i + 1; k2 <= c; k2++) s -= std::conj(L[(size_t)k2 * P + i]) * Ui[(size_t)k2 * P + c];
            Ui[(size_t)i * P + c] = s / std::conj(L[(size_t)i * P + i]);
        }
    return Ui;
}

// The block GMRES iteration with its orthogonalisation on T vectors: the
// Krylov basis Vt [(m+1) P][n], work columns Wt, Tt [P][n]; V (FP64) holds the
// blocks that the preconditioner and operator read, Z their preconditioned
// images.  With T = float2 every new block is converted to FP64 into V.
template <class T>
int gmres_block_impl(Krylov& k, bem_ctx* ctx, const Krylov::Op& op, const double2* B, double2* X, int P, int m,
                     double tol, int max_iter, int* iters, double* relres, bool zero_guess, const Krylov::Op* prec,
                     bool* deficient, T* Vt, T* Wt, T* Tt) {
    constexpr bool F32 = std::is_same<T, float2>::value;
    const int64_t n = k.n, ldk = (int64_t)P * n;
    const unsigned nbl = (unsigned)((ldk + KV_THREADS - 1) / KV_THREADS);
    int rc;
    std::vector<double> bnorm(P), rres(P, 1.0);
    if ((rc = k.norms(ctx, B, P, bnorm.data()))) return rc;
    for (int c = 0; c < P; c++) iters[c] = 0;
    std::vector<double2> tmp((size_t)P * P);
    std::vector<zd> Gh((size_t)P * P);
    // orthonormalise the P columns of Wc in place (column scaling folded into
    // the first of two Cholesky QR passes); Rout: W_in = Q Rout, upper P x P
    auto orth = [&](T* Wc, std::vector<zd>& Rout) -> int {
        std::vector<double> D(P, 1.0);
        std::fill(Rout.begin(), Rout.end(), zd(0));
        for (int c = 0; c < P; c++) Rout[(size_t)c * P + c] = 1.0;
        for (int pass = 0; pass < 2; pass++) {
            const T* src = pass == 0 ? Wc : Tt;
            T* dst = pass == 0 ? Tt : Wc;
            int e = block_dots(ctx, k, src, P, src, P, k.bC);
            if (e) return e;
            CK(cudaMemcpyAsync(tmp.data(), k.bC, tmp.size() * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            for (int c = 0; c < P; c++) {
                const double g = tmp[(size_t)c * P + c].x;
                D[c] = pass == 0 && g > 0 ? std::sqrt(g) : 1.0;
            }
            for (int i = 0; i < P; i++)
                for (int j = 0; j < P; j++)
                    Gh[(size_t)i * P + j] = zd(tmp[(size_t)i * P + j].x, tmp[(size_t)i * P + j].y) / (D[i] * D[j]);
            // dependent columns (the block space is exhausted): a pivot of the
            // column-scaled Gram matrix below 1e-6 (FP32 vectors, whose Gram
            // entries carry errors near 1e-7; singular values below 1e-3 of
            // the largest) or 1e-12 (FP64), where Cholesky QR stops being
            // reliable anyway
            if (!cholesky(Gh, P, F32 ? 1e-6 : 1e-12)) return BEM_ERR_NOT_CONVERGED;
            const std::vector<zd> Ui = upper_inverse(Gh, P);
            for (int i = 0; i < P; i++)
                for (int j = 0; j < P; j++) {
                    const zd v = Ui[(size_t)i * P + j] / D[i];
                    tmp[(size_t)i * P + j] = make_double2(v.real(), v.imag());
                }
            CK(cudaMemcpyAsync(k.bC, tmp.data(), tmp.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
            if ((e = block_combine(ctx, n, src, P, P, k.bC, 1.0, (const T*)nullptr, 0.0, dst))) return e;
            // Rout <- U D Rout
            std::vector<zd> Rt((size_t)P * P);
            for (int i = 0; i < P; i++)
                for (int j = 0; j < P; j++) {
                    zd s = 0;
                    for (int k2 = i; k2 < P; k2++) s += std::conj(Gh[(size_t)k2 * P + i]) * D[k2] * Rout[(size_t)k2 * P + j];
                    Rt[(size_t)i * P + j] = s;
                }
            Rout = Rt;
        }
        return BEM_OK;
    };
    const int KM = (m + 1) * P;
    double2* Hs = k.hs_pin;  // rotated block Hessenberg (upper triangle), Hs[col * KM + row]; pinned, mirrored on the device
    std::vector<double2> Gr((size_t)KM * P);         // rotated right-hand sides, row-major Gr[row * P + c]
    std::vector<double2> rcs((size_t)m * P * P), rsn((size_t)m * P * P);  // P Givens rotations per basis column
    int total = 0;
    bool first = true;
    while (total < max_iter) {
        // block residual into V_0 (and its T copy)
        if (first && zero_guess) {
            CK(cudaMemcpyAsync(k.V, B, (size_t)ldk * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaMemsetAsync(X, 0, (size_t)ldk * sizeof(double2), ctx->stream));
        } else {
            if ((rc = op(X, k.t))) return rc;
            kv_axpby<<<nbl, KV_THREADS, 0, ctx->stream>>>(ldk, make_double2(1, 0), B, make_double2(-1, 0), k.t, k.V);
            ctx->launches += 1;
        }
        first = false;
        std::vector<double> rn(P);
        if ((rc = k.norms(ctx, k.V, P, rn.data()))) return rc;
        bool open = false;
        for (int c = 0; c < P; c++) {
            rres[c] = bnorm[c] > 0 ? rn[c] / bnorm[c] : 0.0;
            open |= rres[c] > tol;
        }
        if (!open) break;
        if constexpr (F32) kv_to32<<<nbl, KV_THREADS, 0, ctx->stream>>>(ldk, k.V, Vt);
        std::vector<zd> S((size_t)P * P);
        if ((rc = orth(Vt, S))) {
            if (rc != BEM_ERR_NOT_CONVERGED) return rc;
            // dependent residual columns: nothing to build on; if this call has
            // made no step yet the caller solves the block another way
            if (total == 0 && deficient) {
                *deficient = true;
                return BEM_OK;
            }
            break;
        }
        if constexpr (F32) kv_to64<<<nbl, KV_THREADS, 0, ctx->stream>>>(ldk, Vt, k.V);
        std::fill(Gr.begin(), Gr.end(), make_double2(0, 0));
        for (int r = 0; r < P; r++)
            for (int c = 0; c < P; c++) Gr[(size_t)r * P + c] = make_double2(S[(size_t)r * P + c].real(), S[(size_t)r * P + c].imag());
        // Step j's device work (preconditioner, operator, CGS2, its coefficients
        // copied to pinned memory) is issued before the host folds step j - 1
        // into the least squares (band Givens, O(j P^3) on the host), so the two
        // overlap; the stopping test therefore lags one step, and a step issued
        // after the last one needed is discarded.
        int folded = 0;        // steps in the least squares
        int issued = 0;        // steps whose device work was issued
        bool breakdown = false, converged = false, pending = false;
        std::vector<zd> Rn_pend((size_t)P * P);
        // the new block column of the Hessenberg matrix, row-major over its P
        // columns (Hb[row * P + c]), plain double arithmetic
        // (a, b) <- (conj(cs) a + conj(sn) b, -sn a + cs b) on rows (row, row + 1) of columns c0..P-1
        auto rot = [&](double2* M, int ld, int row, int c0, int c1, double2 cs, double2 sn) {
            double2* A = M + (size_t)row * ld;
            double2* Bq = M + (size_t)(row + 1) * ld;
            for (int c = c0; c < c1; c++) {
                const double2 a = A[c], b = Bq[c];
                A[c] = make_double2(cs.x * a.x + cs.y * a.y + sn.x * b.x + sn.y * b.y,
                                    cs.x * a.y - cs.y * a.x + sn.x * b.y - sn.y * b.x);
                Bq[c] = make_double2(-(sn.x * a.x - sn.y * a.y) + cs.x * b.x - cs.y * b.y,
                                     -(sn.x * a.y + sn.y * a.x) + cs.x * b.y + cs.y * b.x);
            }
        };
        // fold step jj (coefficients hc, new-block factor Rn); true once every column meets tol
        auto fold = [&](int jj, const double2* hc, const std::vector<zd>& Rn) -> bool {
            const int K = (jj + 1) * P;
            std::vector<double2> Hb((size_t)(K + P) * P);
            for (int kk = 0; kk < K; kk++)
                for (int c = 0; c < P; c++) {
                    const double2 a = hc[(size_t)kk * P + c], b = hc[(size_t)K * P + (size_t)kk * P + c];
                    Hb[(size_t)kk * P + c] = make_double2(a.x + b.x, a.y + b.y);
                }
            for (int r = 0; r < P; r++)
                for (int c = 0; c < P; c++)
                    Hb[(size_t)(K + r) * P + c] = make_double2(Rn[(size_t)r * P + c].real(), Rn[(size_t)r * P + c].imag());
            // earlier rotations (in the order they were made) on all P new columns
            for (int qq = 0; qq < jj * P; qq++)
                for (int l = 0; l < P; l++)
                    rot(Hb.data(), P, qq + P - 1 - l, 0, P, rcs[(size_t)qq * P + l], rsn[(size_t)qq * P + l]);
            // P new rotations per column, applied to the later columns of the block and to G
            for (int c = 0; c < P; c++) {
                const int q = jj * P + c;
                for (int l = 0; l < P; l++) {
                    const int row = q + P - 1 - l;
                    const double2 a = Hb[(size_t)row * P + c], b = Hb[(size_t)(row + 1) * P + c];
                    const double den = std::sqrt(a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
                    const double2 cs = den > 0 ? make_double2(a.x / den, a.y / den) : make_double2(1, 0);
                    const double2 sn = den > 0 ? make_double2(b.x / den, b.y / den) : make_double2(0, 0);
                    rcs[(size_t)q * P + l] = cs;
                    rsn[(size_t)q * P + l] = sn;
                    Hb[(size_t)row * P + c] = make_double2(den, 0);
                    Hb[(size_t)(row + 1) * P + c] = make_double2(0, 0);
                    rot(Hb.data(), P, row, c + 1, P, cs, sn);
                    rot(Gr.data(), P, row, 0, P, cs, sn);
                }
            }
            // keep the rotated columns (upper triangle) for the back substitution,
            // mirrored on the device while the next step runs
            for (int c = 0; c < P; c++) {
                const int q = jj * P + c;
                double2* col = &Hs[(size_t)q * KM];
                for (int r = 0; r <= q; r++) col[r] = Hb[(size_t)r * P + c];
            }
            cudaMemcpyAsync(k.hs_dev + (size_t)jj * P * KM, Hs + (size_t)jj * P * KM, (size_t)P * KM * sizeof(double2),
                            cudaMemcpyHostToDevice, ctx->stream);
            // residual of each column: the last P rows of its rotated right-hand side
            bool all = true;
            for (int c = 0; c < P; c++) {
                double s2 = 0;
                for (int r = K; r < K + P; r++) s2 += Gr[(size_t)r * P + c].x * Gr[(size_t)r * P + c].x +
                                                      Gr[(size_t)r * P + c].y * Gr[(size_t)r * P + c].y;
                rres[c] = bnorm[c] > 0 ? std::sqrt(s2) / bnorm[c] : 0.0;
                if (rres[c] > tol) {
                    all = false;
                    iters[c]++;
                }
            }
            return all;
        };
        while (true) {
            const int j = issued;
            const bool issue = !breakdown && !converged && j < m && total + (pending ? 1 : 0) < max_iter;
            double2* hc = k.hpin + (size_t)(j & 1) * 2 * KM * P;
            if (issue) {
                double2* Vj = k.V + (size_t)j * ldk;
                if (prec) {
                    double2* Zj = k.Z + (size_t)j * ldk;
                    if ((rc = (*prec)(Vj, Zj))) return rc;
                    if ((rc = op(Zj, k.w))) return rc;
                } else if ((rc = op(Vj, k.w))) {
                    return rc;
                }
                if constexpr (F32) kv_to32<<<nbl, KV_THREADS, 0, ctx->stream>>>(ldk, k.w, Wt);
                const int K = (j + 1) * P;
                // CGS2 against every basis vector so far; both coefficient sets read back at once
                for (int pass = 0; pass < 2; pass++) {
                    double2* Cp = k.bC + (size_t)pass * K * P;
                    if ((rc = block_dots(ctx, k, (const T*)Vt, K, (const T*)Wt, P, Cp))) return rc;
                    if ((rc = block_combine(ctx, n, (const T*)Vt, K, P, Cp, -1.0, (const T*)Wt, 1.0, Wt))) return rc;
                }
                CK(cudaMemcpyAsync(hc, k.bC, (size_t)2 * K * P * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
                issued++;
            }
            if (pending) {  // while the GPU works on step j
                pending = false;
                converged = fold(folded, k.hpin + (size_t)(folded & 1) * 2 * KM * P, Rn_pend);
                folded++;
                total++;
                if (converged) break;
            }
            if (!issue) break;
            CK(cudaStreamSynchronize(ctx->stream));
            rc = orth(Wt, Rn_pend);
            if (rc == BEM_ERR_NOT_CONVERGED) {  // the block space is exhausted: solve with what there is
                breakdown = true;
                rc = BEM_OK;
                std::fill(Rn_pend.begin(), Rn_pend.end(), zd(0));
            } else if (rc) {
                return rc;
            } else {
                T* Vn = Vt + (size_t)(j + 1) * ldk;
                CK(cudaMemcpyAsync(Vn, Wt, (size_t)ldk * sizeof(T), cudaMemcpyDeviceToDevice, ctx->stream));
                if constexpr (F32) kv_to64<<<nbl, KV_THREADS, 0, ctx->stream>>>(ldk, Wt, k.V + (size_t)(j + 1) * ldk);
            }
            pending = true;
        }
        const int j = folded;
        // Y = H^-1 G (upper triangular, J unknowns per column), X += Z Y (FP64)
        const int J = j * P;
        if (J > 0) {
            // Y = H^-1 G on the device (H mirrored column by column as it was folded)
            CK(cudaMemcpyAsync(k.gs_dev, Gr.data(), (size_t)J * P * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
            for (int i1 = J; i1 > 0; i1 -= BS_ROWS) {
                const int i0 = std::max(0, i1 - BS_ROWS);
                bs_block_kernel<<<1, dim3((unsigned)P, (unsigned)BS_ROWS), 0, ctx->stream>>>(k.hs_dev, KM, k.gs_dev, k.bC, P,
                                                                                        i0, i1);
                if (i0 > 0)
                    bs_update_kernel<<<(unsigned)(((int64_t)i0 * P + 255) / 256), 256, 0, ctx->stream>>>(
                        k.hs_dev, KM, k.gs_dev, k.bC, P, i0, i1);
                ctx->launches += i0 > 0 ? 2 : 1;
            }
            CK(cudaGetLastError());
            if ((rc = block_combine(ctx, n, (const double2*)(prec ? k.Z : k.V), J, P, k.bC, 1.0, (const double2*)X, 1.0, X)))
                return rc;
        }
        bool open2 = false;
        for (int c = 0; c < P; c++) open2 |= rres[c] > tol;
        if (!open2 || breakdown) break;
    }
    // true residuals of the given systems
    if ((rc = op(X, k.t))) return rc;
    kv_axpby<<<nbl, KV_THREADS, 0, ctx->stream>>>(ldk, make_double2(1, 0), B, make_double2(-1, 0), k.t, k.t);
    ctx->launches += 1;
    std::vector<double> rn(P);
    if ((rc = k.norms(ctx, k.t, P, rn.data()))) return rc;
    for (int c = 0; c < P; c++) relres[c] = bnorm[c] > 0 ? rn[c] / bnorm[c] : 0.0;
    return BEM_OK;
}

}  // namespace

int Krylov::gmres_block(bem_ctx* ctx, const Op& op, const double2* B, double2* X, int64_t Rn, int restart,
                        double tol, int max_iter, int* iters, double* relres, bool zero_guess, const Op* prec,
                        bool fp32_basis, bool* deficient) {
    const int P = (int)Rn;
    if (deficient) *deficient = false;
    int rc = ensure(ctx, n, restart, Rn);
    if (rc) return rc;
    if (prec && (rc = ensure_flexible(ctx))) return rc;
    const int m = restart;
    // scratch: partials of K x P dots (K <= (m+1) P) and two sets of K x P coefficients
    // (FP64: K x P x nsplit <= 8 K P; tiled FP32: K x nsplit <= 64 max(row tiles, 608))
    const size_t gx_max = ((size_t)(m + 1) * P + KD_ROWS - 1) / KD_ROWS;
    const size_t need_part = std::max((size_t)(m + 1) * P * P * 8, (size_t)P * KD_ROWS * std::max<size_t>(gx_max, 608)),
                 need_c = (size_t)2 * (m + 1) * P * P + (size_t)P * P;
    if (bpart_n < need_part) {
        dfree_buf(ctx, (void**)&bpart);
        bpart = (double2*)ctx->dalloc(need_part * sizeof(double2), &rc);
        if (rc) { bpart = nullptr; bpart_n = 0; return rc; }
        bpart_n = need_part;
    }
    // the Hessenberg matrix, pinned on the host and mirrored on the device, and the back substitution's G
    const size_t need_hs = (size_t)(m + 1) * P * m * P;
    if (hs_n < need_hs) {
        if (hs_pin) cudaFreeHost(hs_pin);
        hs_pin = nullptr;
        hs_n = 0;
        dfree_buf(ctx, (void**)&hs_dev);
        dfree_buf(ctx, (void**)&gs_dev);
        if (cudaHostAlloc((void**)&hs_pin, need_hs * sizeof(double2), cudaHostAllocDefault) != cudaSuccess) {
            hs_pin = nullptr;
            return ctx->fail(BEM_ERR_CUDA, "block GMRES: pinned Hessenberg buffer");
        }
        hs_dev = (double2*)ctx->dalloc(need_hs * sizeof(double2), &rc);
        if (rc) { hs_dev = nullptr; return rc; }
        gs_dev = (double2*)ctx->dalloc((size_t)(m + 1) * P * P * sizeof(double2), &rc);
        if (rc) { gs_dev = nullptr; return rc; }
        hs_n = need_hs;
    }
    const size_t need_h = (size_t)2 * 2 * (m + 1) * P * P;  // two steps of two K x P coefficient sets
    if (hpin_n < need_h) {
        if (hpin) cudaFreeHost(hpin);
        hpin = nullptr;
        hpin_n = 0;
        if (cudaHostAlloc((void**)&hpin, need_h * sizeof(double2), cudaHostAllocDefault) != cudaSuccess) {
            hpin = nullptr;
            return ctx->fail(BEM_ERR_CUDA, "block GMRES: pinned host buffer");
        }
        hpin_n = need_h;
    }
    if (bC_n < need_c) {
        dfree_buf(ctx, (void**)&bC);
        bC = (double2*)ctx->dalloc(need_c * sizeof(double2), &rc);
        if (rc) { bC = nullptr; bC_n = 0; return rc; }
        bC_n = need_c;
    }
    if (!fp32_basis)
        return gmres_block_impl<double2>(*this, ctx, op, B, X, P, m, tol, max_iter, iters, relres, zero_guess, prec,
                                         deficient, V, w, t);
    const size_t need32 = (size_t)(m + 3) * P * n;  // basis, then two work blocks
    if (b32_n < need32) {
        dfree_buf(ctx, (void**)&b32);
        b32 = (float2*)ctx->dalloc(need32 * sizeof(float2), &rc);
        if (rc) { b32 = nullptr; b32_n = 0; return rc; }
        b32_n = need32;
    }
    float2* V32 = b32;
    float2* W32 = b32 + (size_t)(m + 1) * P * n;
    float2* T32 = W32 + (size_t)P * n;
    return gmres_block_impl<float2>(*this, ctx, op, B, X, P, m, tol, max_iter, iters, relres, zero_guess, prec,
                                    deficient, V32, W32, T32);
}
