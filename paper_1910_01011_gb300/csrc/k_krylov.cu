// k_krylov.cu -- restarted GMRES with FP64 device vectors (the paper's
// solver: GMRES, restart 100, Sec. 3).  Arnoldi by classical Gram-Schmidt
// applied twice (one batched dot-product kernel and one batched update per
// pass), deterministic fixed-order reductions, Givens rotations on the host
// (the Hessenberg column is j+2 numbers per iteration).
#include <cuda_runtime.h>

#include <algorithm>
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
    return BEM_OK;
}

int Krylov::ensure_flexible(bem_ctx* ctx) {
    if (Z) return BEM_OK;
    int rc;
    Z = (double2*)ctx->dalloc((size_t)m * R * n * sizeof(double2), &rc);
    return rc;
}

void Krylov::release(bem_ctx* ctx) {
    for (void* p : {(void*)V, (void*)w, (void*)t, (void*)part, (void*)h, (void*)y, (void*)sc, (void*)Z}) ctx->dfree(p);
    V = w = t = part = h = y = Z = nullptr;
    sc = nullptr;
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
// given), x holds the initial guess on entry.
int Krylov::gmres(bem_ctx* ctx, const Op& op, const double2* b, double2* x, int restart, double tol, int max_iter,
                  int* iters, double* relres, bool zero_guess, const Op* prec) {
    using cd = std::complex<double>;
    int rc = ensure(ctx, n, restart);
    if (rc) return rc;
    if (prec && (rc = ensure_flexible(ctx))) return rc;
    const int64_t ldz = R * n;  // stride of the flexible basis (column 0 of each block)
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
            if (prec) {
                double2* zj = Z + (int64_t)j * ldz;
                if ((rc = (*prec)(V + (int64_t)j * n, zj))) return rc;
                if ((rc = op(zj, vj1))) return rc;
            } else if ((rc = op(V + (int64_t)j * n, vj1))) {
                return rc;
            }
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
        if (prec) kv_combine<<<nb, KV_THREADS, 0, ctx->stream>>>(Z, ldz, j, y, x, n);
        else kv_combine<<<nb, KV_THREADS, 0, ctx->stream>>>(V, n, j, y, x, n);
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
    using cd = std::complex<double>;
    int rc = ensure(ctx, n, restart, Rn);
    if (rc) return rc;
    if (prec && (rc = ensure_flexible(ctx))) return rc;
    const int64_t ldk = Rn * n;  // stride between basis blocks
    const int ldh = m + 2;
    const unsigned nb = (unsigned)((n + KV_THREADS - 1) / KV_THREADS);
    const dim3 gcol(nb, (unsigned)Rn);
    std::vector<double> bnorm(Rn), beta(Rn), hn(Rn), scale(Rn), res(Rn, 0.0);
    if ((rc = norms(ctx, B, Rn, bnorm.data()))) return rc;
    std::vector<char> live(Rn);
    for (int64_t r = 0; r < Rn; r++) {
        iters[r] = 0;
        live[r] = bnorm[r] > 0;
    }
    const size_t hs = (size_t)(restart + 1) * restart;
    std::vector<cd> H(hs * Rn), cs((size_t)restart * Rn), sn((size_t)restart * Rn), g((size_t)(restart + 1) * Rn);
    std::vector<int> jr(Rn);
    std::vector<char> run(Rn);
    std::vector<double2> hc((size_t)ldh * Rn), hc2((size_t)ldh * Rn), yd((size_t)ldh * Rn);
    int total = 0;
    bool first = true;
    auto upload_scale = [&]() -> int {
        CK(cudaMemcpyAsync(sc, scale.data(), Rn * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        return BEM_OK;
    };
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
        if ((rc = norms(ctx, V, Rn, beta.data()))) return rc;
        bool any = false;
        for (int64_t r = 0; r < Rn; r++) {
            if (live[r]) res[r] = beta[r] / bnorm[r];
            run[r] = live[r] && res[r] > tol;
            live[r] = run[r];
            any |= run[r];
            scale[r] = run[r] ? 1.0 / beta[r] : 0.0;  // finished columns carry zeros
            jr[r] = 0;
            std::fill(g.begin() + (size_t)r * (restart + 1), g.begin() + (size_t)(r + 1) * (restart + 1), cd(0));
            g[(size_t)r * (restart + 1)] = run[r] ? beta[r] : 0.0;
        }
        if (!any) break;
        if ((rc = upload_scale())) return rc;
        kvb_scale<<<gcol, KV_THREADS, 0, ctx->stream>>>(V, n, sc);
        ctx->launches += 1;
        int j = 0;
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
            CK(cudaGetLastError());
            CK(cudaMemcpyAsync(hc.data(), h, hc.size() * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaMemcpyAsync(hc2.data(), y, hc2.size() * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
            if ((rc = norms(ctx, vj1, Rn, hn.data()))) return rc;  // synchronises
            total++;
            bool still = false;
            for (int64_t r = 0; r < Rn; r++) {
                scale[r] = 0.0;
                if (!run[r]) continue;
                cd* Hr = H.data() + hs * r;
                cd* csr = cs.data() + (size_t)restart * r;
                cd* snr = sn.data() + (size_t)restart * r;
                cd* gr = g.data() + (size_t)(restart + 1) * r;
                for (int i = 0; i <= j; i++) {
                    const double2 a = hc[(size_t)r * ldh + i], b2 = hc2[(size_t)r * ldh + i];
                    Hr[(size_t)i * restart + j] = cd(a.x + b2.x, a.y + b2.y);
                }
                Hr[(size_t)(j + 1) * restart + j] = hn[r];
                for (int i = 0; i < j; i++) {
                    const cd a = Hr[(size_t)i * restart + j], c = Hr[(size_t)(i + 1) * restart + j];
                    Hr[(size_t)i * restart + j] = std::conj(csr[i]) * a + std::conj(snr[i]) * c;
                    Hr[(size_t)(i + 1) * restart + j] = -snr[i] * a + csr[i] * c;
                }
                const cd a = Hr[(size_t)j * restart + j], c = Hr[(size_t)(j + 1) * restart + j];
                const double den = std::sqrt(std::norm(a) + std::norm(c));
                csr[j] = den > 0 ? a / den : 1.0;
                snr[j] = den > 0 ? c / den : 0.0;
                Hr[(size_t)j * restart + j] = den;
                Hr[(size_t)(j + 1) * restart + j] = 0;
                gr[j + 1] = -snr[j] * gr[j];
                gr[j] = std::conj(csr[j]) * gr[j];
                iters[r]++;
                jr[r] = j + 1;
                res[r] = std::abs(gr[j + 1]) / bnorm[r];
                if (res[r] <= tol || hn[r] == 0) {
                    run[r] = 0;
                } else {
                    scale[r] = 1.0 / hn[r];
                    still = true;
                }
            }
            if ((rc = upload_scale())) return rc;
            kvb_scale<<<gcol, KV_THREADS, 0, ctx->stream>>>(vj1, n, sc);
            ctx->launches += 1;
            if (!still) {
                j++;
                break;
            }
        }
        // back substitution per column (its own length) and X += V y
        std::fill(yd.begin(), yd.end(), make_double2(0, 0));
        for (int64_t r = 0; r < Rn; r++) {
            const int jj = jr[r];
            const cd* Hr = H.data() + hs * r;
            const cd* gr = g.data() + (size_t)(restart + 1) * r;
            std::vector<cd> yv(jj);
            for (int i = jj - 1; i >= 0; i--) {
                cd s2 = gr[i];
                for (int k = i + 1; k < jj; k++) s2 -= Hr[(size_t)i * restart + k] * yv[k];
                yv[i] = s2 / Hr[(size_t)i * restart + i];
            }
            for (int i = 0; i < jj; i++) yd[(size_t)r * ldh + i] = make_double2(yv[i].real(), yv[i].imag());
        }
        CK(cudaMemcpyAsync(y, yd.data(), yd.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
        if (j > 0) {
            kvb_update<<<gcol, KV_THREADS, 0, ctx->stream>>>(prec ? Z : V, ldk, j, y, ldh, X, n, 1.0);
            ctx->launches += 1;
        }
        CK(cudaGetLastError());
        bool open = false;
        for (int64_t r = 0; r < Rn; r++) open |= live[r] && res[r] > tol;
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
