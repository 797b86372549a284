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

int Krylov::ensure_flexible(bem_ctx* ctx) {
    if (Z) return BEM_OK;
    int rc;
    Z = (double2*)ctx->dalloc((size_t)m * R * n * sizeof(double2), &rc);
    return rc;
}

void Krylov::release(bem_ctx* ctx) {
    for (void* p : {(void*)V, (void*)w, (void*)t, (void*)part, (void*)h, (void*)y, (void*)sc, (void*)Z, (void*)H,
                    (void*)cs, (void*)sn, (void*)g, (void*)bn, (void*)res, (void*)run, (void*)jr, (void*)its,
                    (void*)n_run})
        ctx->dfree(p);
    V = w = t = part = h = y = Z = H = cs = sn = g = nullptr;
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
