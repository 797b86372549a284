// k_sparse.cu -- the OSRC block-diagonal preconditioner (paper Sec. 2.3,
// eqs. OSRC_prec, OSRC_prec_blocks, OSRC_DtN_NtD_maps) on device CSR data.
//
// Per domain j the preconditioner block is diag(DtN, NtD) with
//   DtN ~ i k sqrt(1 + X),  NtD ~ (i k)^-1 (1 + X)^-1/2,  X = Delta_Gamma / k_eps^2,
// the square root replaced by the rotated-branch Pade approximant
//   sqrt(1 + z) ~ C0 + sum_l A_l z / (1 + B_l z)
// and Delta_Gamma by -M^-1 S (P1 mass M and stiffness S on the surface).
// With g = M u:
//   bracket(u) = C0 g - sum_l (A_l / k_eps^2) S (M - (B_l / k_eps^2) S)^-1 g
//   DtN (weak)   = i k bracket(u)
//   NtD (strong) = (i k)^-1 (M - S / k_eps^2)^-1 bracket(u)
// composed with the Galerkin rows in strong form:
//   row1 -> M^-1 DtN(M^-1 row1),   row2 -> NtD(M^-1 row2).
// The sparse systems M - beta S (complex symmetric) are solved by
// Jacobi-preconditioned conjugate-orthogonal CG (COCG), batched over the
// systems of one stage, to a tight relative residual so that the
// preconditioner is a fixed linear map to within that tolerance.
// M and S share the P1 vertex-adjacency pattern; the matrix of a system is
// formed on the fly as M_ij - beta S_ij.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <vector>

#include "ctx.h"
#include "internal.h"

namespace gbem {

constexpr int SP_THREADS = 256;

struct OsrcState {
    int64_t n = 0, nnz = 0;            // global vertex count, nonzeros (block diagonal over domains)
    int64_t* rp = nullptr;             // [n+1]
    int32_t* ci = nullptr;             // [nnz]
    double* vm = nullptr;              // mass values
    double* vs = nullptr;              // stiffness values
    double* dm = nullptr;              // diag(M)
    double* ds = nullptr;              // diag(S)
    int n_pade = 0;
    double2 C0{}, ikk{};               // C0 and i k
    std::vector<double2> A, B;         // A_l / k_eps^2, B_l / k_eps^2
    double2 inv_keps2{};               // 1 / k_eps^2
    int max_sys = 0;
    int nblk = 0;
    // batched COCG state, [max_sys][n] complex
    double2 *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *b = nullptr;
    double2* beta = nullptr;           // [max_sys] shifts
    double* part = nullptr;            // [max_sys][nblk][4] partial sums
    double* scal = nullptr;            // [max_sys][8]: rho(2 parities) re/im, bnorm2, rnorm2, active
    int* flags = nullptr;              // [max_sys] active
    // stage vectors, [2][n] or [2*n_pade][n]
    double2 *u = nullptr, *g = nullptr, *w = nullptr, *br = nullptr;
    double tol = 1e-11;
    int max_iter = 20000;
    long long iters_last = 0;
};

// ---------------------------------------------------------------- kernels

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// Block reduction of NV doubles (fixed order) into out[0..NV).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* out) {
    __shared__ double sh[SP_THREADS / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < NV; k++) {
        double t = v[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[warp][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0;
        for (int w = 0; w < SP_THREADS / 32; w++) t += sh[w][threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

// Sum of part[s][0..nblk)[k] in block order, computed redundantly by every block.
__device__ __forceinline__ double reduce_parts(const double* part, int s, int nblk, int k) {
    __shared__ double sh[SP_THREADS];
    double t = 0;
    for (int b = threadIdx.x; b < nblk; b += SP_THREADS) t += part[((int64_t)s * nblk + b) * 4 + k];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int o = SP_THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

struct CocgArgs {
    int64_t n;
    const int64_t* rp;
    const int32_t* ci;
    const double *vm, *vs, *dm, *ds;
    const double2* beta;
    double2 *x, *r, *z, *p, *q, *b;
    double* part;
    double* scal;
    int nblk;
    int it;
    double tol2;
};

__device__ __forceinline__ double2 diag_inv(const CocgArgs& a, int64_t i, double2 be) {
    const double2 d = make_double2(a.dm[i] - be.x * a.ds[i], -be.y * a.ds[i]);
    return cdiv(make_double2(1.0, 0.0), d);
}

// init: x = 0, r = b, z = D^-1 b, p = z; partials of b^T z and |b|^2
__global__ void cocg_init(CocgArgs a) {
    const int s = blockIdx.y;
    const double2 be = a.beta[s];
    const int64_t off = (int64_t)s * a.n;
    double v[4] = {0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * SP_THREADS) {
        const double2 bi = a.b[off + i];
        const double2 zi = cmul(diag_inv(a, i, be), bi);
        a.x[off + i] = make_double2(0, 0);
        a.r[off + i] = bi;
        a.z[off + i] = zi;
        a.p[off + i] = zi;
        const double2 rz = cmul(bi, zi);
        v[0] += rz.x;
        v[1] += rz.y;
        v[2] += bi.x * bi.x + bi.y * bi.y;
    }
    block_sum<4>(v, a.part + ((int64_t)s * a.nblk + blockIdx.x) * 4);
}

__global__ void cocg_init_scalars(CocgArgs a) {
    const int s = blockIdx.x;
    const double rr = reduce_parts(a.part, s, a.nblk, 0), ri = reduce_parts(a.part, s, a.nblk, 1);
    const double bb = reduce_parts(a.part, s, a.nblk, 2);
    if (threadIdx.x == 0) {
        double* sc = a.scal + (int64_t)s * 8;
        sc[0] = rr; sc[1] = ri;        // rho (parity 0)
        sc[4] = bb;                    // |b|^2
        sc[5] = bb;                    // |r|^2
        sc[6] = (bb > 0) ? 1.0 : 0.0;  // active
    }
}

// q = (M - beta S) p ; partials of p^T q
__global__ void cocg_spmv(CocgArgs a) {
    const int s = blockIdx.y;
    const double2 be = a.beta[s];
    const int64_t off = (int64_t)s * a.n;
    double v[4] = {0, 0, 0, 0};
    const bool active = a.scal[(int64_t)s * 8 + 6] != 0.0;
    if (active)
        for (int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * SP_THREADS) {
            double qr = 0, qi = 0;
            for (int64_t e = a.rp[i]; e < a.rp[i + 1]; e++) {
                const double2 pj = a.p[off + a.ci[e]];
                const double mr = a.vm[e] - be.x * a.vs[e], mi = -be.y * a.vs[e];
                qr += mr * pj.x - mi * pj.y;
                qi += mr * pj.y + mi * pj.x;
            }
            a.q[off + i] = make_double2(qr, qi);
            const double2 pi = a.p[off + i];
            v[0] += pi.x * qr - pi.y * qi;
            v[1] += pi.x * qi + pi.y * qr;
        }
    block_sum<4>(v, a.part + ((int64_t)s * a.nblk + blockIdx.x) * 4);
}

// alpha = rho / (p^T q); x += alpha p; r -= alpha q; z = D^-1 r; partials of r^T z, |r|^2
__global__ void cocg_update(CocgArgs a) {
    const int s = blockIdx.y;
    const double* sc = a.scal + (int64_t)s * 8;
    const bool active = sc[6] != 0.0;
    const double pqr = reduce_parts(a.part, s, a.nblk, 0), pqi = reduce_parts(a.part, s, a.nblk, 1);
    __syncthreads();
    double v[4] = {0, 0, 0, 0};
    if (active) {
        const int par = a.it & 1;
        const double2 rho = make_double2(sc[2 * par], sc[2 * par + 1]);
        const double2 alpha = cdiv(rho, make_double2(pqr, pqi));
        const double2 be = a.beta[s];
        const int64_t off = (int64_t)s * a.n;
        for (int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * SP_THREADS) {
            const double2 pi = a.p[off + i], qi = a.q[off + i];
            double2 xi = a.x[off + i], ri = a.r[off + i];
            const double2 ap = cmul(alpha, pi), aq = cmul(alpha, qi);
            xi.x += ap.x; xi.y += ap.y;
            ri.x -= aq.x; ri.y -= aq.y;
            a.x[off + i] = xi;
            a.r[off + i] = ri;
            const double2 zi = cmul(diag_inv(a, i, be), ri);
            a.z[off + i] = zi;
            const double2 rz = cmul(ri, zi);
            v[0] += rz.x;
            v[1] += rz.y;
            v[2] += ri.x * ri.x + ri.y * ri.y;
        }
    }
    __syncthreads();
    block_sum<4>(v, a.part + ((int64_t)s * a.nblk + blockIdx.x) * 4);
}

// beta = rho_new / rho; p = z + beta p; block 0 stores rho_new and the
// convergence state
__global__ void cocg_direction(CocgArgs a) {
    const int s = blockIdx.y;
    double* sc = a.scal + (int64_t)s * 8;
    const bool active = sc[6] != 0.0;
    const double nr = reduce_parts(a.part, s, a.nblk, 0), ni = reduce_parts(a.part, s, a.nblk, 1);
    const double rr = reduce_parts(a.part, s, a.nblk, 2);
    if (!active) return;
    const int par = a.it & 1;
    const double2 rho = make_double2(sc[2 * par], sc[2 * par + 1]);
    const double2 bt = cdiv(make_double2(nr, ni), rho);
    const int64_t off = (int64_t)s * a.n;
    for (int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * SP_THREADS) {
        const double2 zi = a.z[off + i], pi = a.p[off + i];
        const double2 bp = cmul(bt, pi);
        a.p[off + i] = make_double2(zi.x + bp.x, zi.y + bp.y);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc[2 * (1 - par)] = nr;
        sc[2 * (1 - par) + 1] = ni;
        sc[5] = rr;
    }
}

// After a direction step: deactivate converged systems (run by one thread per system).
__global__ void cocg_check(double* scal, int n_sys, double tol2) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sys) return;
    double* sc = scal + (int64_t)s * 8;
    if (sc[6] != 0.0 && sc[5] <= tol2 * sc[4]) sc[6] = 0.0;
}

// y[s][i] = (M - beta_s S) x[s][i]  (plain SpMV, beta per system)
__global__ void spmv_shift(int64_t n, const int64_t* rp, const int32_t* ci, const double* vm, const double* vs,
                           double2 beta, const double2* x, double2* y) {
    const int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x;
    if (i >= n) return;
    double yr = 0, yi = 0;
    for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
        const double2 xj = x[ci[e]];
        const double mr = vm[e] - beta.x * vs[e], mi = -beta.y * vs[e];
        yr += mr * xj.x - mi * xj.y;
        yi += mr * xj.y + mi * xj.x;
    }
    y[i] = make_double2(yr, yi);
}

// bracket = C0 g - sum_l A_l (S w_l), for the two stage rows at once:
// g: [2][n], w: [2][L][n], out: [2][n]
struct BracketArgs {
    int64_t n;
    const int64_t* rp;
    const int32_t* ci;
    const double* vs;
    const double2* g;
    const double2* w;
    int L;
    double2 C0;
    double2 A[16];
    double2 post[2];   // factor applied to row 0 / row 1 of the result
    double2* out;
};

__global__ void bracket_kernel(BracketArgs a) {
    const int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x;
    const int row = blockIdx.y;
    if (i >= a.n) return;
    double2 acc = cmul(a.C0, a.g[(int64_t)row * a.n + i]);
    for (int l = 0; l < a.L; l++) {
        const double2* wl = a.w + ((int64_t)row * a.L + l) * a.n;
        double sr = 0, si = 0;
        for (int64_t e = a.rp[i]; e < a.rp[i + 1]; e++) {
            const double2 wj = wl[a.ci[e]];
            sr += a.vs[e] * wj.x;
            si += a.vs[e] * wj.y;
        }
        const double2 t = cmul(a.A[l], make_double2(sr, si));
        acc.x -= t.x;
        acc.y -= t.y;
    }
    a.out[(int64_t)row * a.n + i] = cmul(a.post[row], acc);
}

// gather system-order rows into vertex arrays: out[0][v] = y[dof1[v]], out[1][v] = y[dof2[v]]
__global__ void rows_to_vertex(int64_t n, const int64_t* d1, const int64_t* d2, const double2* y, double2* out) {
    const int64_t v = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x;
    if (v >= n) return;
    out[v] = y[d1[v]];
    out[n + v] = y[d2[v]];
}

__global__ void vertex_to_rows(int64_t n, const int64_t* d1, const int64_t* d2, const double2* in0,
                               const double2* in1, double2* y) {
    const int64_t v = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x;
    if (v >= n) return;
    y[d1[v]] = in0[v];
    y[d2[v]] = in1[v];
}

}  // namespace gbem

using namespace gbem;

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// ---------------------------------------------------------------- host set-up

void destroy_osrc_state(bem_ctx* ctx) {
    delete ctx->osrc;
    ctx->osrc = nullptr;
    ctx->osrc_ready = false;
}

static int osrc_build(bem_ctx* ctx) {
    if (ctx->osrc_ready) return BEM_OK;
    int rc = ctx->finalize();
    if (rc) return rc;
    const Geometry& g = ctx->geo;
    OsrcState* o = ctx->osrc;
    if (!o) {
        o = new OsrcState();
        ctx->osrc = o;
    } else {
        for (void* p : {(void*)o->rp, (void*)o->ci, (void*)o->vm, (void*)o->vs, (void*)o->dm, (void*)o->ds,
                        (void*)o->x, (void*)o->r, (void*)o->z, (void*)o->p, (void*)o->q, (void*)o->b,
                        (void*)o->beta, (void*)o->part, (void*)o->scal, (void*)o->u, (void*)o->g, (void*)o->w,
                        (void*)o->br})
            ctx->dfree(p);
        *o = OsrcState();
    }
    // P1 mass and stiffness in one CSR pattern (per domain, block diagonal)
    const int64_t n = g.n_vert;
    std::vector<std::map<int32_t, std::pair<double, double>>> rows(n);
    for (int64_t s = 0; s < g.n_slots; s++) {
        if (g.slot_v[4 * s] < 0) continue;
        const double A = g.slot_area[s];
        double grad[3][3];
        // grad lambda_k = curl_k x n (surface curl = n x grad)
        for (int k = 0; k < 3; k++) {
            const double* c = &g.slot_curl[9 * s + 3 * k];
            const double* nn = &g.slot_n[3 * s];
            grad[k][0] = c[1] * nn[2] - c[2] * nn[1];
            grad[k][1] = c[2] * nn[0] - c[0] * nn[2];
            grad[k][2] = c[0] * nn[1] - c[1] * nn[0];
        }
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                const double m = A * (a == b ? 2.0 : 1.0) / 12.0;
                const double st = A * (grad[a][0] * grad[b][0] + grad[a][1] * grad[b][1] + grad[a][2] * grad[b][2]);
                auto& e = rows[g.slot_v[4 * s + a]][g.slot_v[4 * s + b]];
                e.first += m;
                e.second += st;
            }
    }
    std::vector<int64_t> rp(n + 1, 0);
    std::vector<int32_t> ci;
    std::vector<double> vm, vs, dm(n), ds(n);
    for (int64_t i = 0; i < n; i++) {
        for (auto& kv : rows[i]) {
            ci.push_back(kv.first);
            vm.push_back(kv.second.first);
            vs.push_back(kv.second.second);
            if (kv.first == i) {
                dm[i] = kv.second.first;
                ds[i] = kv.second.second;
            }
        }
        rp[i + 1] = (int64_t)ci.size();
    }
    o->n = n;
    o->nnz = (int64_t)ci.size();
    auto up = [&](auto** dst, const auto& v) -> int {
        using T = typename std::remove_reference<decltype(v)>::type::value_type;
        *dst = (T*)ctx->dalloc(std::max<size_t>(1, v.size()) * sizeof(T), &rc);
        if (rc) return rc;
        cudaError_t e = cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, ctx->stream);
        return e == cudaSuccess ? BEM_OK : ctx->fail(BEM_ERR_CUDA, "osrc upload");
    };
    if ((rc = up(&o->rp, rp)) || (rc = up(&o->ci, ci)) || (rc = up(&o->vm, vm)) || (rc = up(&o->vs, vs)) ||
        (rc = up(&o->dm, dm)) || (rc = up(&o->ds, ds)))
        return rc;
    // Pade coefficients and the damped wavenumber (exterior k0, Sec. 2.3)
    const int N = ctx->opts.n_pade;
    if (N < 1 || N > 16) return ctx->fail(BEM_ERR_INVALID_ARG, "n_pade must be in 1..16");
    const double th = ctx->opts.pade_theta;
    using cd = std::complex<double>;
    const cd e = std::exp(cd(0, -th));
    cd R = 1.0;
    std::vector<double> al(N), bl(N);
    for (int l = 1; l <= N; l++) {
        const double s = std::sin(l * M_PI / (2 * N + 1)), c = std::cos(l * M_PI / (2 * N + 1));
        al[l - 1] = 2.0 / (2 * N + 1) * s * s;
        bl[l - 1] = c * c;
        R += al[l - 1] * (e - 1.0) / (1.0 + bl[l - 1] * (e - 1.0));
    }
    const cd C0 = std::exp(cd(0, 0.5 * th)) * R;
    double reps = ctx->opts.r_eps > 0 ? ctx->opts.r_eps : 0.1 * g.max_diameter;
    const cd k0(ctx->k0re, ctx->k0im);
    const double eps = 0.4 * std::pow(ctx->k0re, ctx->opts.eps_exponent) * std::pow(reps, -2.0 / 3.0);
    const cd keps = k0 + cd(0, eps);
    const cd ik2 = 1.0 / (keps * keps);
    o->n_pade = N;
    o->C0 = make_double2(C0.real(), C0.imag());
    const cd ik = cd(0, 1) * k0;
    o->ikk = make_double2(ik.real(), ik.imag());
    o->inv_keps2 = make_double2(ik2.real(), ik2.imag());
    o->A.resize(N);
    o->B.resize(N);
    for (int l = 0; l < N; l++) {
        const cd den = 1.0 + bl[l] * (e - 1.0);
        const cd Al = std::exp(cd(0, -0.5 * th)) * al[l] / (den * den) * ik2;
        const cd Bl = e * bl[l] / den * ik2;
        o->A[l] = make_double2(Al.real(), Al.imag());
        o->B[l] = make_double2(Bl.real(), Bl.imag());
    }
    // batched state
    o->max_sys = std::max(2 * N, 2);
    o->nblk = (int)std::min<int64_t>(128, (n + SP_THREADS - 1) / SP_THREADS);
    const size_t vec = (size_t)o->max_sys * n * sizeof(double2);
    o->x = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->r = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->z = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->p = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->q = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->b = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->beta = (double2*)ctx->dalloc(o->max_sys * sizeof(double2), &rc); if (rc) return rc;
    o->part = (double*)ctx->dalloc((size_t)o->max_sys * o->nblk * 4 * sizeof(double), &rc); if (rc) return rc;
    o->scal = (double*)ctx->dalloc((size_t)o->max_sys * 8 * sizeof(double), &rc); if (rc) return rc;
    o->u = (double2*)ctx->dalloc(2 * n * sizeof(double2), &rc); if (rc) return rc;
    o->g = (double2*)ctx->dalloc(2 * n * sizeof(double2), &rc); if (rc) return rc;
    o->w = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->br = (double2*)ctx->dalloc(2 * n * sizeof(double2), &rc); if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->osrc_ready = true;
    return BEM_OK;
}

// Solve (M - beta_s S) x_s = b_s for s < n_sys (b already in o->b, shifts
// in o->beta); solutions in o->x.
static int cocg_solve(bem_ctx* ctx, int n_sys) {
    OsrcState* o = ctx->osrc;
    CocgArgs a{};
    a.n = o->n; a.rp = o->rp; a.ci = o->ci; a.vm = o->vm; a.vs = o->vs; a.dm = o->dm; a.ds = o->ds;
    a.beta = o->beta; a.x = o->x; a.r = o->r; a.z = o->z; a.p = o->p; a.q = o->q; a.b = o->b;
    a.part = o->part; a.scal = o->scal; a.nblk = o->nblk; a.tol2 = o->tol * o->tol;
    const dim3 grid(o->nblk, n_sys);
    cocg_init<<<grid, SP_THREADS, 0, ctx->stream>>>(a);
    cocg_init_scalars<<<n_sys, SP_THREADS, 0, ctx->stream>>>(a);
    ctx->launches += 2;
    std::vector<double> sc(8 * n_sys);
    int it = 0;
    for (; it < o->max_iter;) {
        for (int k = 0; k < 32; k++, it++) {
            a.it = it;
            cocg_spmv<<<grid, SP_THREADS, 0, ctx->stream>>>(a);
            cocg_update<<<grid, SP_THREADS, 0, ctx->stream>>>(a);
            cocg_direction<<<grid, SP_THREADS, 0, ctx->stream>>>(a);
            cocg_check<<<(n_sys + 31) / 32, 32, 0, ctx->stream>>>(o->scal, n_sys, a.tol2);
            ctx->launches += 4;
        }
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(sc.data(), o->scal, sc.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        bool any = false;
        for (int s = 0; s < n_sys; s++) any |= sc[8 * s + 6] != 0.0;
        if (!any) break;
    }
    o->iters_last += it;
    for (int s = 0; s < n_sys; s++)
        if (sc[8 * s + 6] != 0.0)
            return ctx->fail(BEM_ERR_NOT_CONVERGED, "OSRC inner COCG solve did not converge");
    return BEM_OK;
}

// y = P x for Galerkin rows x (system order); both device vectors.
// With u = M^-1 row, the bracket's g = M u is the row itself, so the Pade
// solves take the rows directly: 2 N_pade + 2 sparse solves per application.
int bem_ctx::apply_prec(const double2* xin, double2* yout) {
    bem_ctx* const ctx = this;
    int rc = osrc_build(this);
    if (rc) return rc;
    OsrcState* o = osrc;
    const int64_t n = o->n;
    const unsigned nb = (unsigned)((n + SP_THREADS - 1) / SP_THREADS);
    const int L = o->n_pade;
    // rows in vertex order: g[0] = row1, g[1] = row2
    rows_to_vertex<<<nb, SP_THREADS, 0, stream>>>(n, dev.v_dof1, dev.v_dof2, xin, o->g);
    // Pade solves w_{i,l} = (M - B_l S)^-1 row_i, systems ordered [row][l]
    std::vector<double2> be(o->max_sys, make_double2(0, 0));
    for (int row = 0; row < 2; row++)
        for (int l = 0; l < L; l++) {
            CK(cudaMemcpyAsync(o->b + ((int64_t)row * L + l) * n, o->g + (int64_t)row * n, n * sizeof(double2),
                               cudaMemcpyDeviceToDevice, stream));
            be[row * L + l] = o->B[l];
        }
    CK(cudaMemcpyAsync(o->beta, be.data(), 2 * L * sizeof(double2), cudaMemcpyHostToDevice, stream));
    if ((rc = cocg_solve(this, 2 * L))) return rc;
    // brackets; row 1 scaled by i k (the DtN weak form)
    BracketArgs ba{};
    ba.n = n; ba.rp = o->rp; ba.ci = o->ci; ba.vs = o->vs; ba.g = o->g; ba.w = o->x; ba.L = L; ba.C0 = o->C0;
    for (int l = 0; l < L; l++) ba.A[l] = o->A[l];
    ba.post[0] = o->ikk;
    ba.post[1] = make_double2(1.0, 0.0);
    ba.out = o->b;
    bracket_kernel<<<dim3(nb, 2), SP_THREADS, 0, stream>>>(ba);
    // out1 = M^-1 (i k bracket_1);  out2 = (M - S/k_eps^2)^-1 bracket_2, then / (i k)
    be[0] = make_double2(0, 0);
    be[1] = o->inv_keps2;
    CK(cudaMemcpyAsync(o->beta, be.data(), 2 * sizeof(double2), cudaMemcpyHostToDevice, stream));
    if ((rc = cocg_solve(this, 2))) return rc;
    const std::complex<double> inv = 1.0 / std::complex<double>(o->ikk.x, o->ikk.y);
    BracketArgs cp{};  // scaled copy (no Pade terms): u_row = post_row * x_row
    cp.n = n; cp.rp = o->rp; cp.ci = o->ci; cp.vs = o->vs; cp.g = o->x; cp.w = nullptr; cp.L = 0;
    cp.C0 = make_double2(1.0, 0.0);
    cp.post[0] = make_double2(1.0, 0.0);
    cp.post[1] = make_double2(inv.real(), inv.imag());
    cp.out = o->u;
    bracket_kernel<<<dim3(nb, 2), SP_THREADS, 0, stream>>>(cp);
    vertex_to_rows<<<nb, SP_THREADS, 0, stream>>>(n, dev.v_dof1, dev.v_dof2, o->u, o->u + n, yout);
    launches += 4;
    CK(cudaGetLastError());
    return BEM_OK;
}

int bem_ctx::apply_prec_ahat(const double2* x, double2* y, int precision) {
    int rc = apply_ahat(x, dev.ys2, precision);
    if (rc) return rc;
    return apply_prec(dev.ys2, y);
}
