// k_krylov.cu -- restarted GMRES with FP64 device vectors (the paper's
// solver: GMRES, restart 100, Sec. 3).  Arnoldi by classical Gram-Schmidt
// applied twice (one batched dot-product kernel and one batched update per
// pass), deterministic fixed-order reductions, Givens rotations on the host
// (the Hessenberg column is j+2 numbers per iteration).
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <functional>
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

}  // namespace gbem

using namespace gbem;

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int Krylov::ensure(bem_ctx* ctx, int64_t n_, int m_) {
    if (n == n_ && m >= m_) return BEM_OK;
    release(ctx);
    n = n_;
    m = m_;
    int rc;
    V = (double2*)ctx->dalloc((size_t)(m + 1) * n * sizeof(double2), &rc); if (rc) return rc;
    w = (double2*)ctx->dalloc(n * sizeof(double2), &rc); if (rc) return rc;
    t = (double2*)ctx->dalloc(n * sizeof(double2), &rc); if (rc) return rc;
    part = (double2*)ctx->dalloc((size_t)(m + 2) * KV_BLOCKS * sizeof(double2), &rc); if (rc) return rc;
    h = (double2*)ctx->dalloc((m + 2) * sizeof(double2), &rc); if (rc) return rc;
    y = (double2*)ctx->dalloc((m + 2) * sizeof(double2), &rc); if (rc) return rc;
    return BEM_OK;
}

void Krylov::release(bem_ctx* ctx) {
    for (void* p : {(void*)V, (void*)w, (void*)t, (void*)part, (void*)h, (void*)y}) ctx->dfree(p);
    V = w = t = part = h = y = nullptr;
    n = 0;
    m = 0;
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
                  double2* out) {
    const unsigned nb = (unsigned)((n + KV_THREADS - 1) / KV_THREADS);
    kv_axpby<<<nb, KV_THREADS, 0, ctx->stream>>>(n, make_double2(a.real(), a.imag()), x,
                                                 make_double2(b.real(), b.imag()), z, out);
    ctx->launches += 1;
    CK(cudaGetLastError());
    return BEM_OK;
}

// Solve op(x) = b to ||b - op(x)|| <= tol ||b|| (residual of the system it is
// given), x holds the initial guess on entry.
int Krylov::gmres(bem_ctx* ctx, const std::function<int(const double2*, double2*)>& op, const double2* b,
                  double2* x, int restart, double tol, int max_iter, int* iters, double* relres,
                  bool zero_guess) {
    using cd = std::complex<double>;
    int rc = ensure(ctx, n, restart);
    if (rc) return rc;
    const unsigned nb = (unsigned)((n + KV_THREADS - 1) / KV_THREADS);
    double bnorm;
    if ((rc = norm(ctx, b, &bnorm))) return rc;
    *iters = 0;
    if (bnorm == 0) {
        CK(cudaMemsetAsync(x, 0, n * sizeof(double2), ctx->stream));
        *relres = 0;
        return BEM_OK;
    }
    std::vector<cd> H((size_t)(restart + 1) * restart), cs(restart), sn(restart), g(restart + 1);
    std::vector<double2> hcol(restart + 2);
    double res = 1.0;
    bool first = true;
    while (*iters < max_iter) {
        // r = b - op(x) into V_0
        if (first && zero_guess) {
            CK(cudaMemcpyAsync(V, b, n * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaMemsetAsync(x, 0, n * sizeof(double2), ctx->stream));
        } else {
            if ((rc = op(x, t))) return rc;
            if ((rc = axpby(ctx, 1.0, b, -1.0, t, V))) return rc;
        }
        first = false;
        double beta;
        if ((rc = norm(ctx, V, &beta))) return rc;
        res = beta / bnorm;
        if (res <= tol) break;
        if ((rc = axpby(ctx, 1.0 / beta, V, 0.0, nullptr, V))) return rc;
        std::fill(g.begin(), g.end(), cd(0));
        g[0] = beta;
        int j = 0;
        for (; j < restart && *iters < max_iter; j++) {
            double2* vj1 = V + (int64_t)(j + 1) * n;
            if ((rc = op(V + (int64_t)j * n, vj1))) return rc;
            // CGS2: two passes of h = V^H w; w -= V h
            for (int pass = 0; pass < 2; pass++) {
                kv_dots<<<dim3(KV_BLOCKS, j + 1), KV_THREADS, 0, ctx->stream>>>(V, n, j + 1, vj1, n, part);
                kv_reduce<<<j + 1, 32, 0, ctx->stream>>>(part, KV_BLOCKS, pass == 0 ? h : y, 0);
                kv_subtract<<<nb, KV_THREADS, 0, ctx->stream>>>(V, n, j + 1, pass == 0 ? h : y, vj1, n);
                ctx->launches += 3;
            }
            CK(cudaGetLastError());
            double hn;
            if ((rc = norm(ctx, vj1, &hn))) return rc;
            CK(cudaMemcpyAsync(hcol.data(), h, (j + 1) * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
            std::vector<double2> h2(j + 1);
            CK(cudaMemcpyAsync(h2.data(), y, (j + 1) * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            for (int i = 0; i <= j; i++) H[(size_t)i * restart + j] = cd(hcol[i].x + h2[i].x, hcol[i].y + h2[i].y);
            H[(size_t)(j + 1) * restart + j] = hn;
            if (hn > 0) {
                if ((rc = axpby(ctx, 1.0 / hn, vj1, 0.0, nullptr, vj1))) return rc;
            }
            // apply previous rotations, then the new one
            for (int i = 0; i < j; i++) {
                cd a = H[(size_t)i * restart + j], c = H[(size_t)(i + 1) * restart + j];
                H[(size_t)i * restart + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * c;
                H[(size_t)(i + 1) * restart + j] = -sn[i] * a + cs[i] * c;
            }
            cd a = H[(size_t)j * restart + j], c = H[(size_t)(j + 1) * restart + j];
            double den = std::sqrt(std::norm(a) + std::norm(c));
            cs[j] = den > 0 ? a / den : 1.0;
            sn[j] = den > 0 ? c / den : 0.0;
            H[(size_t)j * restart + j] = den;
            H[(size_t)(j + 1) * restart + j] = 0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = std::conj(cs[j]) * g[j];
            (*iters)++;
            res = std::abs(g[j + 1]) / bnorm;
            if (res <= tol || hn == 0) {
                j++;
                break;
            }
        }
        // back substitution and x += V y
        std::vector<cd> yv(j);
        for (int i = j - 1; i >= 0; i--) {
            cd s = g[i];
            for (int k = i + 1; k < j; k++) s -= H[(size_t)i * restart + k] * yv[k];
            yv[i] = s / H[(size_t)i * restart + i];
        }
        std::vector<double2> yd(j);
        for (int i = 0; i < j; i++) yd[i] = make_double2(yv[i].real(), yv[i].imag());
        CK(cudaMemcpyAsync(y, yd.data(), j * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
        kv_combine<<<nb, KV_THREADS, 0, ctx->stream>>>(V, n, j, y, x, n);
        ctx->launches += 1;
        CK(cudaGetLastError());
        if (res <= tol) break;
    }
    // true residual of the given system
    if ((rc = op(x, t))) return rc;
    if ((rc = axpby(ctx, 1.0, b, -1.0, t, t))) return rc;
    double rn;
    if ((rc = norm(ctx, t, &rn))) return rc;
    *relres = rn / bnorm;
    return BEM_OK;
}
