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
#include <cooperative_groups.h>
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
    // per domain d (the block's wavenumber k_d, bem_opts.osrc_wavenumber):
    double2 C0{};                      // C0 (the same for every domain)
    std::vector<double2> ikk;          // [n_dom] i k_d
    std::vector<double2> A, B;         // [n_dom][n_pade] A_l / k_eps,d^2, B_l / k_eps,d^2
    std::vector<double2> inv_keps2;    // [n_dom] 1 / k_eps,d^2
    double2* dA = nullptr;             // device [n_dom][n_pade] copy of A
    double2* post_b = nullptr;         // device [n_dom][2]: (i k_d, 1), the bracket rows' factors
    double2* post_c = nullptr;         // device [n_dom][2]: (1, 1 / (i k_d)), the closing factors
    int32_t* vdom = nullptr;           // device [n] domain of each vertex
    int max_sys = 0;
    int64_t max_rhs = 0;               // right-hand sides the batched buffers hold
    int nblk = 0;
    // batched COCG state, [max_sys][n] complex; max_sys = 2 n_pade max_rhs
    double2 *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *b = nullptr;
    double2* beta = nullptr;           // shifts of the systems being solved: beta_pade or beta_close
    double2* beta_pade = nullptr;      // [max_sys][n_dom] Pade shifts B_{s mod n_pade} of each domain
    double2* beta_close = nullptr;     // [2 max_rhs][n_dom] closing systems: 0 and 1 / k_eps^2 alternately
    double* part = nullptr;            // [max_sys][nblk][4] partial sums
    double* scal = nullptr;            // [max_sys][8]: rho(2 parities) re/im, bnorm2, rnorm2, active
    // stage vectors, [max_rhs][2][n]
    double2 *u = nullptr, *g = nullptr;
    double tol = 1e-11;
    int max_iter = 20000;
    long long iters_last = 0;
    // one-CTA-per-(system, domain) solver: domain vertex ranges, status words
    int n_dom = 0;
    int64_t max_dom_nv = 0;
    int ell_w = 0;                     // ELL width (max nonzeros per row), 0 if too wide
    int32_t* ell_ci = nullptr;         // [ell_w][n] column indices (padding: the row itself)
    double *ell_m = nullptr, *ell_s = nullptr;  // [ell_w][n] mass / stiffness values (padding: 0)
    // FP32 copies for the loose solves inside a flexible GMRES (GB300's FP64 rate
    // is ~1/64 of its FP32 rate, and a 10-30 % residual needs no FP64)
    float *ell_m32 = nullptr, *ell_s32 = nullptr, *dm32 = nullptr, *ds32 = nullptr;
    float2 *x32 = nullptr, *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr;  // [max_sys][n]
    int64_t* dom_v0 = nullptr;         // [n_dom + 1] vertex offsets
    unsigned long long* stat = nullptr;  // [0]: iterations (sum over CTAs), [1]: CTAs that did not converge
    // CUDA graphs of GRAPH_ITERS COCG iterations, per (number of systems, tolerance, shift table)
    struct Graph {
        int n_sys;
        double tol;
        const double2* beta;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
    cudaStream_t cap = nullptr;
};

constexpr int GRAPH_ITERS = 32;

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
    const double2* beta;   // [n_sys][nd]
    const int32_t* vdom;   // [n] domain of each row
    int nd;
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
    const double2* bes = a.beta + (int64_t)s * a.nd;
    const int64_t off = (int64_t)s * a.n;
    double v[4] = {0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * SP_THREADS) {
        const double2 bi = a.b[off + i];
        const double2 zi = cmul(diag_inv(a, i, bes[a.vdom[i]]), bi);
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
        sc[7] = 0.0;                   // broken down
    }
}

// q = (M - beta S) p ; partials of p^T q
__global__ void cocg_spmv(CocgArgs a) {
    const int s = blockIdx.y;
    const double2* bes = a.beta + (int64_t)s * a.nd;
    const int64_t off = (int64_t)s * a.n;
    double v[4] = {0, 0, 0, 0};
    const bool active = a.scal[(int64_t)s * 8 + 6] != 0.0;
    if (active)
        for (int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * SP_THREADS) {
            const double2 be = bes[a.vdom[i]];  // the matrix is block diagonal over domains
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
    const int par0 = a.it & 1;
    const double2 alpha0 = cdiv(make_double2(sc[2 * par0], sc[2 * par0 + 1]), make_double2(pqr, pqi));
    const bool finite = isfinite(alpha0.x) && isfinite(alpha0.y);
    if (active && !finite && blockIdx.x == 0 && threadIdx.x == 0) {
        // breakdown (p^T A p = 0): this system stops with its current x
        double* scw = a.scal + (int64_t)s * 8;
        scw[6] = 0.0;
        scw[7] = 1.0;
    }
    if (active && finite) {
        const int par = a.it & 1;
        const double2 rho = make_double2(sc[2 * par], sc[2 * par + 1]);
        const double2 alpha = cdiv(rho, make_double2(pqr, pqi));
        const double2* bes = a.beta + (int64_t)s * a.nd;
        const int64_t off = (int64_t)s * a.n;
        for (int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * SP_THREADS) {
            const double2 pi = a.p[off + i], qi = a.q[off + i];
            double2 xi = a.x[off + i], ri = a.r[off + i];
            const double2 ap = cmul(alpha, pi), aq = cmul(alpha, qi);
            xi.x += ap.x; xi.y += ap.y;
            ri.x -= aq.x; ri.y -= aq.y;
            a.x[off + i] = xi;
            a.r[off + i] = ri;
            const double2 zi = cmul(diag_inv(a, i, bes[a.vdom[i]]), ri);
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
    if (!isfinite(bt.x) || !isfinite(bt.y)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            sc[6] = 0.0;
            sc[7] = 1.0;
        }
        return;
    }
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

// ---- one CTA per (system, domain)
//
// M and S are block diagonal over the domains (P1 functions of one surface
// only couple within it), so every (system, domain) pair is an independent
// complex-symmetric system that one CTA can iterate on its own: the vectors
// of a domain stay in L2, the dot products are CTA reductions, and no
// iteration needs a launch, a grid-wide synchronisation or a host round trip.
// Each CTA stops on its own relative residual |r_j| <= tol |b_j|, so a
// system converges to tol on every domain (hence also globally); after
// max_iter iterations it stops and counts itself in stat[1].
struct CocgCtaArgs {
    int64_t n;                 // vertices (vector length per system)
    const int32_t* eci;        // ELL [W][n]
    const double *em, *es;     // ELL [W][n]
    const double *dm, *ds;
    const double2* beta;       // [n_sys][n_dom]
    const double2* b;          // [n_sys][n]
    double2 *x, *r, *z, *p, *q;
    const int64_t* dom_v0;     // [n_dom + 1]
    int n_dom;
    double tol2;
    int max_iter;
    unsigned long long* stat;
};

// Sum of NV doubles over the CTA; every thread gets the same result (fixed order).
template <int NT, int NV>
__device__ __forceinline__ void cta_sum(double (&v)[NV]) {
    __shared__ double sh[NT / 32][NV];
    __shared__ double tot[NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double t = v[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[warp][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0;
        for (int w = 0; w < NT / 32; w++) t += sh[w][threadIdx.x];
        tot[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = tot[k];
    __syncthreads();  // tot and sh are reused by the next call
}

// Rows a thread handles together: U rows NT apart, so that the loads of all
// U rows (W coalesced ELL entries each) are in flight at once.
constexpr int CTA_U = 4;

template <int NT, int W>
__global__ void __launch_bounds__(NT) cocg_cta_kernel(CocgCtaArgs a) {
    const int s = blockIdx.x / a.n_dom, j = blockIdx.x % a.n_dom;
    const int64_t v0 = a.dom_v0[j], v1 = a.dom_v0[j + 1];
    const int64_t n = a.n, off = (int64_t)s * n;
    const double2 be = a.beta[(int64_t)s * a.n_dom + j];
    const double2* b = a.b + off;
    double2 *x = a.x + off, *r = a.r + off, *z = a.z + off, *p = a.p + off, *q = a.q + off;
    auto dinv = [&](int64_t i) {
        return cdiv(make_double2(1.0, 0.0), make_double2(a.dm[i] - be.x * a.ds[i], -be.y * a.ds[i]));
    };
    // x = 0, r = b, z = D^-1 b, p = z; rho = r^T z, |b|^2
    double v3[3] = {0, 0, 0};
    for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
        const double2 bi = b[i];
        const double2 zi = cmul(dinv(i), bi);
        x[i] = make_double2(0, 0);
        r[i] = bi;
        z[i] = zi;
        p[i] = zi;
        const double2 rz = cmul(bi, zi);
        v3[0] += rz.x;
        v3[1] += rz.y;
        v3[2] += bi.x * bi.x + bi.y * bi.y;
    }
    cta_sum<NT, 3>(v3);
    double2 rho = make_double2(v3[0], v3[1]);
    const double lim = a.tol2 * v3[2];
    if (!(v3[2] > 0)) return;  // zero right-hand side: x = 0
    int it = 0;
    bool ok = false;
    while (it < a.max_iter) {
        it++;
        // q = (M - beta S) p, p^T q
        double v2[2] = {0, 0};
        for (int64_t i0 = v0 + threadIdx.x; i0 < v1; i0 += CTA_U * NT) {
            double qr[CTA_U], qi[CTA_U];
#pragma unroll
            for (int u = 0; u < CTA_U; u++) {
                qr[u] = 0;
                qi[u] = 0;
                const int64_t i = i0 + (int64_t)u * NT;
                if (i < v1) {
#pragma unroll
                    for (int k = 0; k < W; k++) {
                        const int64_t e = (int64_t)k * n + i;
                        const double2 pj = p[a.eci[e]];
                        const double mr = a.em[e] - be.x * a.es[e], mi = -be.y * a.es[e];
                        qr[u] += mr * pj.x - mi * pj.y;
                        qi[u] += mr * pj.y + mi * pj.x;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < CTA_U; u++) {
                const int64_t i = i0 + (int64_t)u * NT;
                if (i < v1) {
                    q[i] = make_double2(qr[u], qi[u]);
                    const double2 pi = p[i];
                    v2[0] += pi.x * qr[u] - pi.y * qi[u];
                    v2[1] += pi.x * qi[u] + pi.y * qr[u];
                }
            }
        }
        cta_sum<NT, 2>(v2);
        const double2 alpha = cdiv(rho, make_double2(v2[0], v2[1]));
        if (!isfinite(alpha.x) || !isfinite(alpha.y)) break;  // breakdown (p^T A p = 0): keep x
        // x += alpha p, r -= alpha q, z = D^-1 r; r^T z, |r|^2
        double w3[3] = {0, 0, 0};
        for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
            const double2 pi = p[i], qi = q[i];
            double2 xi = x[i], ri = r[i];
            const double2 ap = cmul(alpha, pi), aq = cmul(alpha, qi);
            xi.x += ap.x; xi.y += ap.y;
            ri.x -= aq.x; ri.y -= aq.y;
            x[i] = xi;
            r[i] = ri;
            const double2 zi = cmul(dinv(i), ri);
            z[i] = zi;
            const double2 rz = cmul(ri, zi);
            w3[0] += rz.x;
            w3[1] += rz.y;
            w3[2] += ri.x * ri.x + ri.y * ri.y;
        }
        cta_sum<NT, 3>(w3);
        if (w3[2] <= lim) {
            ok = true;
            break;
        }
        const double2 rn = make_double2(w3[0], w3[1]);
        const double2 bt = cdiv(rn, rho);
        if (!isfinite(bt.x) || !isfinite(bt.y)) break;  // breakdown (r^T z = 0 before): keep x
        rho = rn;
        for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
            const double2 zi = z[i], pi = p[i];
            const double2 bp = cmul(bt, pi);
            p[i] = make_double2(zi.x + bp.x, zi.y + bp.y);
        }
        __syncthreads();  // p is read across rows by the next product
    }
    if (threadIdx.x == 0) {
        atomicAdd(&a.stat[0], (unsigned long long)it);
        if (!ok) atomicAdd(&a.stat[1], 1ull);
    }
}

// ---- one thread-block cluster per (system, domain)
//
// For a few systems the one-CTA solver leaves most SMs idle and the
// grid-wide kernels pay four launches per iteration.  Here the CL CTAs of a
// cluster (on CL SMs) share one (system, domain): each owns a contiguous
// slice of the domain's rows, the three reductions of an iteration go through
// distributed shared memory (each CTA writes its partial sums, the cluster
// barrier publishes them, every CTA adds the CL partials in rank order, so all
// CTAs hold bit-identical scalars and take identical branches), and the
// barrier after the direction update makes the new p visible to the other
// CTAs' products (read through L2).  Every CTA of a cluster executes the same
// sequence of cluster barriers: the loop bounds and exits depend only on
// those shared scalars and on max_iter.
constexpr int CL = 8;
// Whether the automatic choice groups the Pade shifts of a right-hand side in
// one cluster.  It does not: on the 41k-triangle rib scene the grouped kernel
// (176 registers, one CTA per SM) took 16.4 / 49.2 / 88.1 ms per application
// to 1 / 8 / 16 right-hand sides against 6.4 / 26.7 / 50.8 ms for one cluster
// per system; the p gathers, not the shared matrix loads, set the pace.
constexpr bool SHIFT_GROUPS_AUTO = false;

namespace cg = cooperative_groups;

template <int NT, int NV>
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cl, double (&v)[NV], double (*buf)[NV], int& phase) {
    __shared__ double sh[NT / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double t = v[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[warp][k] = t;
    }
    __syncthreads();
    double* mine = buf[phase];
    if (threadIdx.x < NV) {
        double t = 0;
        for (int w = 0; w < NT / 32; w++) t += sh[w][threadIdx.x];
        mine[threadIdx.x] = t;
    }
    cl.sync();  // publishes every CTA's partial sums (release / acquire at cluster scope)
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double t = 0;
        for (int r = 0; r < CL; r++) t += cl.map_shared_rank(mine, r)[k];
        v[k] = t;
    }
    phase ^= 1;  // the next sum writes the other buffer, so no second barrier is needed
}

template <int NT, int W>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT) cocg_cluster_kernel(CocgCtaArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double buf2[2][2], buf3[2][3];
    int ph2 = 0, ph3 = 0;
    const int item = blockIdx.x / CL, rank = (int)cl.block_rank();
    const int s = item / a.n_dom, j = item % a.n_dom;
    const int64_t d0 = a.dom_v0[j], d1 = a.dom_v0[j + 1];
    const int64_t per = (d1 - d0 + CL - 1) / CL;
    const int64_t v0 = min(d1, d0 + rank * per), v1 = min(d1, v0 + per);
    const int64_t n = a.n, off = (int64_t)s * n;
    const double2 be = a.beta[(int64_t)s * a.n_dom + j];
    const double2* b = a.b + off;
    double2 *x = a.x + off, *r = a.r + off, *z = a.z + off, *p = a.p + off, *q = a.q + off;
    auto dinv = [&](int64_t i) {
        return cdiv(make_double2(1.0, 0.0), make_double2(a.dm[i] - be.x * a.ds[i], -be.y * a.ds[i]));
    };
    double v3[3] = {0, 0, 0};
    for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
        const double2 bi = b[i];
        const double2 zi = cmul(dinv(i), bi);
        x[i] = make_double2(0, 0);
        r[i] = bi;
        z[i] = zi;
        p[i] = zi;
        const double2 rz = cmul(bi, zi);
        v3[0] += rz.x;
        v3[1] += rz.y;
        v3[2] += bi.x * bi.x + bi.y * bi.y;
    }
    cluster_sum<NT, 3>(cl, v3, buf3, ph3);  // also publishes the initial p
    double2 rho = make_double2(v3[0], v3[1]);
    const double lim = a.tol2 * v3[2];
    int it = 0;
    bool ok = !(v3[2] > 0);  // zero right-hand side: x = 0 is exact
    while (!ok && it < a.max_iter) {
        it++;
        double v2[2] = {0, 0};
        for (int64_t i0 = v0 + threadIdx.x; i0 < v1; i0 += CTA_U * NT) {
            double qr[CTA_U], qi[CTA_U];
#pragma unroll
            for (int u = 0; u < CTA_U; u++) {
                qr[u] = 0;
                qi[u] = 0;
                const int64_t i = i0 + (int64_t)u * NT;
                if (i < v1) {
#pragma unroll
                    for (int k = 0; k < W; k++) {
                        const int64_t e = (int64_t)k * n + i;
                        const double2 pj = __ldcg(p + a.eci[e]);  // other CTAs' rows: read through L2
                        const double mr = a.em[e] - be.x * a.es[e], mi = -be.y * a.es[e];
                        qr[u] += mr * pj.x - mi * pj.y;
                        qi[u] += mr * pj.y + mi * pj.x;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < CTA_U; u++) {
                const int64_t i = i0 + (int64_t)u * NT;
                if (i < v1) {
                    q[i] = make_double2(qr[u], qi[u]);
                    const double2 pi = p[i];
                    v2[0] += pi.x * qr[u] - pi.y * qi[u];
                    v2[1] += pi.x * qi[u] + pi.y * qr[u];
                }
            }
        }
        cluster_sum<NT, 2>(cl, v2, buf2, ph2);
        const double2 alpha = cdiv(rho, make_double2(v2[0], v2[1]));
        if (!isfinite(alpha.x) || !isfinite(alpha.y)) break;  // breakdown, identical in every CTA: keep x
        double w3[3] = {0, 0, 0};
        for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
            const double2 pi = p[i], qi = q[i];
            double2 xi = x[i], ri = r[i];
            const double2 ap = cmul(alpha, pi), aq = cmul(alpha, qi);
            xi.x += ap.x; xi.y += ap.y;
            ri.x -= aq.x; ri.y -= aq.y;
            x[i] = xi;
            r[i] = ri;
            const double2 zi = cmul(dinv(i), ri);
            z[i] = zi;
            const double2 rz = cmul(ri, zi);
            w3[0] += rz.x;
            w3[1] += rz.y;
            w3[2] += ri.x * ri.x + ri.y * ri.y;
        }
        cluster_sum<NT, 3>(cl, w3, buf3, ph3);
        if (w3[2] <= lim) {
            ok = true;
            break;
        }
        const double2 rn = make_double2(w3[0], w3[1]);
        const double2 bt = cdiv(rn, rho);
        if (!isfinite(bt.x) || !isfinite(bt.y)) break;
        rho = rn;
        for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
            const double2 zi = z[i], pi = p[i];
            const double2 bp = cmul(bt, pi);
            p[i] = make_double2(zi.x + bp.x, zi.y + bp.y);
        }
        cl.sync();  // the new p, read across CTAs by the next product
    }
    // no CTA may leave while another still reads its shared memory
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
        atomicAdd(&a.stat[0], (unsigned long long)it);
        if (!ok) atomicAdd(&a.stat[1], 1ull);
    }
}

// ---- the same two solvers in FP32, for loose tolerances
//
// Inside the flexible GMRES the sparse solves stop at a 10-30 % relative
// residual.  In FP64 the cluster solver is bound by GB300's FP64 pipe (68 %
// of its cycles busy on the 41k-triangle rib scene at 16 right-hand sides,
// ncu), so these variants keep the vectors, matrix values and arithmetic in
// FP32: b is read once in FP64, x is written back once in FP64.  The
// iteration, its stopping test and its breakdown guards are those of the FP64
// solvers.

__device__ __forceinline__ float2 fcmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 fcdiv(float2 a, float2 b) {
    const float d = b.x * b.x + b.y * b.y;
    return make_float2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

struct CocgArgs32 {
    int64_t n;
    const int32_t* eci;       // ELL [W][n]
    const float *em, *es;     // ELL [W][n]
    const float *dm, *ds;
    const double2* beta;      // [n_sys][n_dom]
    const double2* b;         // [n_sys][n]
    double2* xout;            // [n_sys][n]
    float2 *x, *r, *z, *p, *q;
    const int64_t* dom_v0;
    int n_dom;
    float tol2;
    int max_iter;
    unsigned long long* stat;
};

template <int NT, int NV>
__device__ __forceinline__ void cta_sum32(float (&v)[NV]) {
    __shared__ float sh[NT / 32][NV];
    __shared__ float tot[NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        float t = v[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[warp][k] = t;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        float t = 0;
        for (int w = 0; w < NT / 32; w++) t += sh[w][threadIdx.x];
        tot[threadIdx.x] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = tot[k];
    __syncthreads();
}

template <int NT>
struct CtaRed32 {
    template <int NV>
    __device__ __forceinline__ void sum(float (&v)[NV]) { cta_sum32<NT, NV>(v); }
    __device__ __forceinline__ void sync() { __syncthreads(); }
};

// Rows [v0, v1) of domain j of system s; `red` sums over the rows of all the
// CTAs that share the system (one CTA, or the CTAs of a cluster).
template <int NT, int W, class Red>
__device__ __forceinline__ void cocg32_body(const CocgArgs32& a, int s, int j, int64_t v0, int64_t v1, Red& red,
                                            bool leader) {
    const int64_t n = a.n, off = (int64_t)s * n;
    const double2 be64 = a.beta[(int64_t)s * a.n_dom + j];
    const float2 be = make_float2((float)be64.x, (float)be64.y);
    const double2* b = a.b + off;
    float2 *x = a.x + off, *r = a.r + off, *z = a.z + off, *p = a.p + off, *q = a.q + off;
    auto dinv = [&](int64_t i) {
        return fcdiv(make_float2(1.f, 0.f), make_float2(a.dm[i] - be.x * a.ds[i], -be.y * a.ds[i]));
    };
    float v3[3] = {0, 0, 0};
    for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
        const double2 b64 = b[i];
        const float2 bi = make_float2((float)b64.x, (float)b64.y);
        const float2 zi = fcmul(dinv(i), bi);
        x[i] = make_float2(0.f, 0.f);
        r[i] = bi;
        z[i] = zi;
        p[i] = zi;
        const float2 rz = fcmul(bi, zi);
        v3[0] += rz.x;
        v3[1] += rz.y;
        v3[2] += bi.x * bi.x + bi.y * bi.y;
    }
    red.template sum<3>(v3);  // also publishes the initial p
    float2 rho = make_float2(v3[0], v3[1]);
    const float lim = a.tol2 * v3[2];
    int it = 0;
    bool ok = !(v3[2] > 0);  // zero right-hand side: x = 0 is exact
    while (!ok && it < a.max_iter) {
        it++;
        float v2[2] = {0, 0};
        for (int64_t i0 = v0 + threadIdx.x; i0 < v1; i0 += CTA_U * NT) {
            float qr[CTA_U], qi[CTA_U];
#pragma unroll
            for (int u = 0; u < CTA_U; u++) {
                qr[u] = 0;
                qi[u] = 0;
                const int64_t i = i0 + (int64_t)u * NT;
                if (i < v1) {
#pragma unroll
                    for (int k = 0; k < W; k++) {
                        const int64_t e = (int64_t)k * n + i;
                        const float2 pj = __ldcg(p + a.eci[e]);  // other CTAs' rows: read through L2
                        const float mr = a.em[e] - be.x * a.es[e], mi = -be.y * a.es[e];
                        qr[u] += mr * pj.x - mi * pj.y;
                        qi[u] += mr * pj.y + mi * pj.x;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < CTA_U; u++) {
                const int64_t i = i0 + (int64_t)u * NT;
                if (i < v1) {
                    q[i] = make_float2(qr[u], qi[u]);
                    const float2 pi = p[i];
                    v2[0] += pi.x * qr[u] - pi.y * qi[u];
                    v2[1] += pi.x * qi[u] + pi.y * qr[u];
                }
            }
        }
        red.template sum<2>(v2);
        const float2 alpha = fcdiv(rho, make_float2(v2[0], v2[1]));
        if (!isfinite(alpha.x) || !isfinite(alpha.y)) break;  // breakdown, identical for every CTA: keep x
        float w3[3] = {0, 0, 0};
        for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
            const float2 pi = p[i], qi = q[i];
            float2 xi = x[i], ri = r[i];
            const float2 ap = fcmul(alpha, pi), aq = fcmul(alpha, qi);
            xi.x += ap.x; xi.y += ap.y;
            ri.x -= aq.x; ri.y -= aq.y;
            x[i] = xi;
            r[i] = ri;
            const float2 zi = fcmul(dinv(i), ri);
            z[i] = zi;
            const float2 rz = fcmul(ri, zi);
            w3[0] += rz.x;
            w3[1] += rz.y;
            w3[2] += ri.x * ri.x + ri.y * ri.y;
        }
        red.template sum<3>(w3);
        if (w3[2] <= lim) {
            ok = true;
            break;
        }
        const float2 rn = make_float2(w3[0], w3[1]);
        const float2 bt = fcdiv(rn, rho);
        if (!isfinite(bt.x) || !isfinite(bt.y)) break;
        rho = rn;
        for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
            const float2 zi = z[i], pi = p[i];
            const float2 bp = fcmul(bt, pi);
            p[i] = make_float2(zi.x + bp.x, zi.y + bp.y);
        }
        red.sync();  // the new p, read across rows (and CTAs) by the next product
    }
    double2* xo = a.xout + off;
    for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) xo[i] = make_double2((double)x[i].x, (double)x[i].y);
    if (leader) {
        atomicAdd(&a.stat[0], (unsigned long long)it);
        if (!ok) atomicAdd(&a.stat[1], 1ull);
    }
}

// At most 64 registers (1024 / NT CTAs of NT threads per SM): the FP32 state
// is small, and the solve's time is the iteration latency of many systems.
template <int NT, int W>
__global__ void __launch_bounds__(NT, 1024 / NT) cocg_cta32_kernel(CocgArgs32 a) {
    const int s = blockIdx.x / a.n_dom, j = blockIdx.x % a.n_dom;
    CtaRed32<NT> red;
    cocg32_body<NT, W>(a, s, j, a.dom_v0[j], a.dom_v0[j + 1], red, threadIdx.x == 0);
}

template <int NT, int NV>
__device__ __forceinline__ void cluster_sum32(cg::cluster_group& cl, float (&v)[NV], float (*buf)[NV], int& phase) {
    __shared__ float sh[NT / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        float t = v[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[warp][k] = t;
    }
    __syncthreads();
    float* mine = buf[phase];
    if (threadIdx.x < NV) {
        float t = 0;
        for (int w = 0; w < NT / 32; w++) t += sh[w][threadIdx.x];
        mine[threadIdx.x] = t;
    }
    cl.sync();  // publishes every CTA's partial sums
#pragma unroll
    for (int k = 0; k < NV; k++) {
        float t = 0;
        for (int r = 0; r < CL; r++) t += cl.map_shared_rank(mine, r)[k];
        v[k] = t;
    }
    phase ^= 1;  // the next sum writes the other buffer
}

template <int NT>
struct ClusterRed32 {
    cg::cluster_group cl;
    float (*buf2)[2];
    float (*buf3)[3];
    int ph2 = 0, ph3 = 0;
    template <int NV>
    __device__ __forceinline__ void sum(float (&v)[NV]) {
        if constexpr (NV == 2) cluster_sum32<NT, 2>(cl, v, buf2, ph2);
        else cluster_sum32<NT, 3>(cl, v, buf3, ph3);
    }
    __device__ __forceinline__ void sync() { cl.sync(); }
};

template <int NT, int W>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT, 1024 / NT) cocg_cluster32_kernel(CocgArgs32 a) {
    __shared__ float buf2[2][2], buf3[2][3];
    ClusterRed32<NT> red{cg::this_cluster(), buf2, buf3};
    const int item = blockIdx.x / CL, rank = (int)red.cl.block_rank();
    const int s = item / a.n_dom, j = item % a.n_dom;
    const int64_t d0 = a.dom_v0[j], d1 = a.dom_v0[j + 1];
    const int64_t per = (d1 - d0 + CL - 1) / CL;
    const int64_t v0 = min(d1, d0 + rank * per), v1 = min(d1, v0 + per);
    cocg32_body<NT, W>(a, s, j, v0, v1, red, rank == 0 && threadIdx.x == 0);
    red.sync();  // no CTA may leave while another still reads its shared memory
}

// ---- the Pade shifts of one right-hand side together: one cluster per (group, domain)
//
// The 2 N_pade Pade systems of a right-hand side come in groups of N_pade
// that share the right-hand side (one row of the bracket) and the matrices,
// differing only in the shift B_l.  One cluster iterates all L shifts of a
// group at once: every ELL entry of M and S is loaded once for the L
// products, the reductions of the L systems travel together, and there are L
// times fewer clusters to schedule.  Each shift is still its own COCG (its
// own alpha, beta and stopping test); a shift that has converged or broken
// down stops changing x, while the others go on.  The shared scalars live in
// shared memory, identical in every CTA of the cluster.

// As cluster_sum, but the NV totals go to shared memory (res[NV]) instead of registers.
template <int NT, int NV>
__device__ __forceinline__ void cluster_sum_to(cg::cluster_group& cl, const double (&v)[NV], double (*buf)[NV],
                                               int& phase, double* res) {
    __shared__ double sh[NT / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double t = v[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh[warp][k] = t;
    }
    __syncthreads();
    double* mine = buf[phase];
    if (threadIdx.x < NV) {
        double t = 0;
        for (int w = 0; w < NT / 32; w++) t += sh[w][threadIdx.x];
        mine[threadIdx.x] = t;
    }
    cl.sync();
    if (threadIdx.x < NV) {
        double t = 0;
        for (int r = 0; r < CL; r++) t += cl.map_shared_rank(mine, r)[threadIdx.x];
        res[threadIdx.x] = t;
    }
    __syncthreads();
    phase ^= 1;
}

template <int NT, int W, int L>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT) cocg_cluster_shift_kernel(CocgCtaArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double bufA[2][2 * L], bufB[2][3 * L];
    __shared__ double resA[2 * L], resB[3 * L];
    __shared__ double2 rho[L], alpha[L], bt[L];
    __shared__ double lim[L];
    __shared__ double2 be[L];
    __shared__ int act[L], brk[L];
    int phA = 0, phB = 0;
    const int item = blockIdx.x / CL, rank = (int)cl.block_rank();
    const int grp = item / a.n_dom, j = item % a.n_dom;
    const int64_t d0 = a.dom_v0[j], d1 = a.dom_v0[j + 1];
    const int64_t per = (d1 - d0 + CL - 1) / CL;
    const int64_t v0 = min(d1, d0 + rank * per), v1 = min(d1, v0 + per);
    const int64_t n = a.n, off0 = (int64_t)grp * L * n;  // system grp*L + l at off0 + l*n
    const double2* b = a.b + off0;                       // the shared right-hand side (first shift's copy)
    if (threadIdx.x < L) {
        be[threadIdx.x] = a.beta[((int64_t)grp * L + threadIdx.x) * a.n_dom + j];
        brk[threadIdx.x] = 0;
    }
    __syncthreads();
    // x = 0, r = b, z = D_l^-1 b, p = z; per shift r^T z, and |b|^2
    {
        double v[3 * L];
#pragma unroll
        for (int t = 0; t < 3 * L; t++) v[t] = 0;
        for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
            const double2 bi = b[i];
#pragma unroll
            for (int l = 0; l < L; l++) {
                const int64_t o = off0 + l * n + i;
                const double2 zi = cmul(cdiv(make_double2(1.0, 0.0),
                                             make_double2(a.dm[i] - be[l].x * a.ds[i], -be[l].y * a.ds[i])), bi);
                a.x[o] = make_double2(0, 0);
                a.r[o] = bi;
                a.z[o] = zi;
                a.p[o] = zi;
                const double2 rz = cmul(bi, zi);
                v[3 * l] += rz.x;
                v[3 * l + 1] += rz.y;
                v[3 * l + 2] += bi.x * bi.x + bi.y * bi.y;
            }
        }
        cluster_sum_to<NT, 3 * L>(cl, v, bufB, phB, resB);  // also publishes the initial p
    }
    if (threadIdx.x < L) {
        const int l = threadIdx.x;
        rho[l] = make_double2(resB[3 * l], resB[3 * l + 1]);
        lim[l] = a.tol2 * resB[3 * l + 2];
        act[l] = resB[3 * l + 2] > 0;
    }
    __syncthreads();
    int it = 0, open = 0;
    for (int l = 0; l < L; l++) open += act[l];
    while (open > 0 && it < a.max_iter) {
        it++;
        // q_l = (M - beta_l S) p_l and p_l^T q_l, every shift from one pass over the ELL entries
        double v2[2 * L];
#pragma unroll
        for (int t = 0; t < 2 * L; t++) v2[t] = 0;
        for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
            double qr[L], qi[L];
#pragma unroll
            for (int l = 0; l < L; l++) qr[l] = qi[l] = 0;
#pragma unroll
            for (int k = 0; k < W; k++) {
                const int64_t e = (int64_t)k * n + i;
                const int64_t c = a.eci[e];
                const double m = a.em[e], sv = a.es[e];
#pragma unroll
                for (int l = 0; l < L; l++) {
                    const double2 pj = __ldcg(a.p + off0 + l * n + c);  // other CTAs' rows: read through L2
                    const double mr = m - be[l].x * sv, mi = -be[l].y * sv;
                    qr[l] += mr * pj.x - mi * pj.y;
                    qi[l] += mr * pj.y + mi * pj.x;
                }
            }
#pragma unroll
            for (int l = 0; l < L; l++) {
                const int64_t o = off0 + l * n + i;
                a.q[o] = make_double2(qr[l], qi[l]);
                const double2 pi = a.p[o];
                v2[2 * l] += pi.x * qr[l] - pi.y * qi[l];
                v2[2 * l + 1] += pi.x * qi[l] + pi.y * qr[l];
            }
        }
        cluster_sum_to<NT, 2 * L>(cl, v2, bufA, phA, resA);
        if (threadIdx.x < L) {
            const int l = threadIdx.x;
            alpha[l] = cdiv(rho[l], make_double2(resA[2 * l], resA[2 * l + 1]));
            if (act[l] && (!isfinite(alpha[l].x) || !isfinite(alpha[l].y))) {
                act[l] = 0;  // breakdown: keep x
                brk[l] = 1;
            }
        }
        __syncthreads();
        double v3[3 * L];
#pragma unroll
        for (int t = 0; t < 3 * L; t++) v3[t] = 0;
        for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
#pragma unroll
            for (int l = 0; l < L; l++) {
                if (!act[l]) continue;
                const int64_t o = off0 + l * n + i;
                const double2 pi = a.p[o], qi = a.q[o];
                double2 xi = a.x[o], ri = a.r[o];
                const double2 ap = cmul(alpha[l], pi), aq = cmul(alpha[l], qi);
                xi.x += ap.x; xi.y += ap.y;
                ri.x -= aq.x; ri.y -= aq.y;
                a.x[o] = xi;
                a.r[o] = ri;
                const double2 zi = cmul(cdiv(make_double2(1.0, 0.0),
                                             make_double2(a.dm[i] - be[l].x * a.ds[i], -be[l].y * a.ds[i])), ri);
                a.z[o] = zi;
                const double2 rz = cmul(ri, zi);
                v3[3 * l] += rz.x;
                v3[3 * l + 1] += rz.y;
                v3[3 * l + 2] += ri.x * ri.x + ri.y * ri.y;
            }
        }
        cluster_sum_to<NT, 3 * L>(cl, v3, bufB, phB, resB);
        if (threadIdx.x < L) {
            const int l = threadIdx.x;
            if (act[l]) {
                if (resB[3 * l + 2] <= lim[l]) {
                    act[l] = 0;  // converged
                } else {
                    const double2 rn = make_double2(resB[3 * l], resB[3 * l + 1]);
                    bt[l] = cdiv(rn, rho[l]);
                    if (!isfinite(bt[l].x) || !isfinite(bt[l].y)) {
                        act[l] = 0;
                        brk[l] = 1;
                    }
                    rho[l] = rn;
                }
            }
        }
        __syncthreads();
        open = 0;
        for (int l = 0; l < L; l++) open += act[l];
        if (open == 0) break;
        for (int64_t i = v0 + threadIdx.x; i < v1; i += NT) {
#pragma unroll
            for (int l = 0; l < L; l++) {
                if (!act[l]) continue;
                const int64_t o = off0 + l * n + i;
                const double2 zi = a.z[o], pi = a.p[o];
                const double2 bp = cmul(bt[l], pi);
                a.p[o] = make_double2(zi.x + bp.x, zi.y + bp.y);
            }
        }
        cl.sync();  // the new p, read across CTAs by the next product
    }
    cl.sync();  // no CTA may leave while another still reads its shared memory
    if (rank == 0 && threadIdx.x == 0) {
        atomicAdd(&a.stat[0], (unsigned long long)it);
        // shifts still open hit the iteration cap; broken-down ones count too
        int bad = 0;
        for (int l = 0; l < L; l++) bad += act[l] || brk[l];
        if (bad) atomicAdd(&a.stat[1], 1ull);
    }
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
    const double2* A;      // [n_dom][L] (vertex i uses the row of its domain)
    const double2* post;   // [n_dom][2] factor applied to row 0 / row 1 of the result
    const int32_t* vdom;   // [n]
    double2* out;
};

// Right-hand side rb = blockIdx.z of a batch: g, out at [rb][2][n], w at [rb][2][L][n].
__global__ void bracket_kernel(BracketArgs a) {
    const int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x;
    const int row = blockIdx.y;
    const int64_t rr = (int64_t)blockIdx.z * 2 + row;  // (rhs, row)
    if (i >= a.n) return;
    const int d = a.vdom[i];
    double2 acc = cmul(a.C0, a.g[rr * a.n + i]);
    for (int l = 0; l < a.L; l++) {
        const double2* wl = a.w + (rr * a.L + l) * a.n;
        double sr = 0, si = 0;
        for (int64_t e = a.rp[i]; e < a.rp[i + 1]; e++) {
            const double2 wj = wl[a.ci[e]];
            sr += a.vs[e] * wj.x;
            si += a.vs[e] * wj.y;
        }
        const double2 t = cmul(a.A[d * a.L + l], make_double2(sr, si));
        acc.x -= t.x;
        acc.y -= t.y;
    }
    a.out[rr * a.n + i] = cmul(a.post[2 * d + row], acc);
}

// gather system-order rows (right-hand side blockIdx.y, N = 2n dofs each) into
// vertex arrays: out[rb][0][v] = y[rb][dof1[v]], out[rb][1][v] = y[rb][dof2[v]]
__global__ void rows_to_vertex(int64_t n, const int64_t* d1, const int64_t* d2, const double2* y, double2* out) {
    const int64_t v = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x;
    const int64_t rb = blockIdx.y;
    if (v >= n) return;
    out[rb * 2 * n + v] = y[rb * 2 * n + d1[v]];
    out[rb * 2 * n + n + v] = y[rb * 2 * n + d2[v]];
}

__global__ void vertex_to_rows(int64_t n, const int64_t* d1, const int64_t* d2, const double2* in, double2* y) {
    const int64_t v = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x;
    const int64_t rb = blockIdx.y;
    if (v >= n) return;
    y[rb * 2 * n + d1[v]] = in[rb * 2 * n + v];
    y[rb * 2 * n + d2[v]] = in[rb * 2 * n + n + v];
}

// Pade right-hand sides: b[(rr L + l)][i] = g[rr][i] for every (rhs, row) pair rr
__global__ void replicate_rows(int64_t n, int L, const double2* g, double2* b) {
    const int64_t i = (int64_t)blockIdx.x * SP_THREADS + threadIdx.x;
    const int64_t sys = blockIdx.y;  // rr * L + l
    if (i >= n) return;
    b[sys * n + i] = g[(sys / L) * n + i];
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
    if (ctx->osrc) {
        for (auto& g : ctx->osrc->graphs) cudaGraphExecDestroy(g.exec);
        if (ctx->osrc->cap) cudaStreamDestroy(ctx->osrc->cap);
    }
    delete ctx->osrc;
    ctx->osrc = nullptr;
    ctx->osrc_ready = false;
}

// Batched buffers for R right-hand sides (2 n_pade R systems); captured
// graphs hold the old pointers and are dropped when the buffers move.
static int ensure_osrc_batch(bem_ctx* ctx, OsrcState* o, int64_t R) {
    if (R <= o->max_rhs) return BEM_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    for (void* p : {(void*)o->x, (void*)o->r, (void*)o->z, (void*)o->p, (void*)o->q, (void*)o->b, (void*)o->beta_pade,
                    (void*)o->beta_close, (void*)o->part, (void*)o->scal, (void*)o->u, (void*)o->g, (void*)o->x32,
                    (void*)o->r32, (void*)o->z32, (void*)o->p32, (void*)o->q32})
        ctx->dfree(p);
    o->x = o->r = o->z = o->p = o->q = o->b = o->beta = o->beta_pade = o->beta_close = o->u = o->g = nullptr;
    o->x32 = o->r32 = o->z32 = o->p32 = o->q32 = nullptr;
    o->part = o->scal = nullptr;
    for (auto& gr : o->graphs) cudaGraphExecDestroy(gr.exec);
    o->graphs.clear();
    o->max_rhs = 0;
    o->max_sys = 0;
    const int64_t n = o->n;
    const int64_t ms = 2 * (int64_t)o->n_pade * R;
    if (ms > 65535) return ctx->fail(BEM_ERR_INVALID_ARG, "too many right-hand sides for one preconditioner batch");
    int rc;
    const size_t vec = (size_t)ms * n * sizeof(double2);
    o->x = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->r = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->z = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->p = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->q = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->b = (double2*)ctx->dalloc(vec, &rc); if (rc) return rc;
    o->beta_pade = (double2*)ctx->dalloc((size_t)ms * o->n_dom * sizeof(double2), &rc); if (rc) return rc;
    o->beta_close = (double2*)ctx->dalloc((size_t)2 * R * o->n_dom * sizeof(double2), &rc); if (rc) return rc;
    {
        // the shift tables, for every batch up to R (both repeat per right-hand side)
        const int nd = o->n_dom, L = o->n_pade;
        std::vector<double2> bp((size_t)ms * nd), bc((size_t)2 * R * nd);
        for (int64_t s = 0; s < ms; s++)
            for (int d = 0; d < nd; d++) bp[(size_t)s * nd + d] = o->B[(size_t)d * L + s % L];
        for (int64_t rb = 0; rb < R; rb++)
            for (int d = 0; d < nd; d++) {
                bc[(size_t)(2 * rb) * nd + d] = make_double2(0, 0);
                bc[(size_t)(2 * rb + 1) * nd + d] = o->inv_keps2[d];
            }
        CK(cudaMemcpyAsync(o->beta_pade, bp.data(), bp.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(o->beta_close, bc.data(), bc.size() * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    o->part = (double*)ctx->dalloc((size_t)ms * o->nblk * 4 * sizeof(double), &rc); if (rc) return rc;
    o->scal = (double*)ctx->dalloc((size_t)ms * 8 * sizeof(double), &rc); if (rc) return rc;
    o->u = (double2*)ctx->dalloc((size_t)2 * R * n * sizeof(double2), &rc); if (rc) return rc;
    o->g = (double2*)ctx->dalloc((size_t)2 * R * n * sizeof(double2), &rc); if (rc) return rc;
    const size_t vec32 = (size_t)ms * n * sizeof(float2);
    for (float2** v : {&o->x32, &o->r32, &o->z32, &o->p32, &o->q32}) {
        *v = (float2*)ctx->dalloc(vec32, &rc);
        if (rc) return rc;
    }
    o->max_sys = (int)ms;
    o->max_rhs = R;
    return BEM_OK;
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
                        (void*)o->beta, (void*)o->part, (void*)o->scal, (void*)o->u, (void*)o->g,
                        (void*)o->dom_v0, (void*)o->stat, (void*)o->ell_ci, (void*)o->ell_m, (void*)o->ell_s,
                        (void*)o->dA, (void*)o->post_b, (void*)o->post_c, (void*)o->vdom, (void*)o->ell_m32,
                        (void*)o->ell_s32, (void*)o->dm32, (void*)o->ds32, (void*)o->x32, (void*)o->r32,
                        (void*)o->z32, (void*)o->p32, (void*)o->q32})
            ctx->dfree(p);
        for (auto& g : o->graphs) cudaGraphExecDestroy(g.exec);
        if (o->cap) cudaStreamDestroy(o->cap);
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
    // ELL copy of the pattern for the one-CTA solver (width = most nonzeros in a row)
    int64_t wmax = 0;
    for (int64_t i = 0; i < n; i++) wmax = std::max(wmax, rp[i + 1] - rp[i]);
    const int ell_w = wmax <= 8 ? 8 : wmax <= 12 ? 12 : wmax <= 16 ? 16 : 0;
    std::vector<int32_t> eci;
    std::vector<double> em, es;
    if (ell_w) {
        eci.assign((size_t)ell_w * n, 0);
        em.assign((size_t)ell_w * n, 0.0);
        es.assign((size_t)ell_w * n, 0.0);
        for (int64_t i = 0; i < n; i++)
            for (int k = 0; k < ell_w; k++) {
                const int64_t e = rp[i] + k;
                const size_t d = (size_t)k * n + i;
                if (e < rp[i + 1]) {
                    eci[d] = ci[e];
                    em[d] = vm[e];
                    es[d] = vs[e];
                } else {
                    eci[d] = (int32_t)i;
                }
            }
    }
    o->ell_w = ell_w;
    std::vector<int64_t> dv0(g.n_dom + 1, 0);
    for (int d = 0; d < g.n_dom; d++) {
        dv0[d + 1] = g.dom_vert_off[d] + g.dom_nv[d];
        o->max_dom_nv = std::max(o->max_dom_nv, g.dom_nv[d]);
    }
    o->n_dom = g.n_dom;
    std::vector<unsigned long long> st0(2, 0ull);
    if ((rc = up(&o->rp, rp)) || (rc = up(&o->ci, ci)) || (rc = up(&o->vm, vm)) || (rc = up(&o->vs, vs)) ||
        (rc = up(&o->dm, dm)) || (rc = up(&o->ds, ds)) || (rc = up(&o->dom_v0, dv0)) || (rc = up(&o->stat, st0)))
        return rc;
    if (ell_w && ((rc = up(&o->ell_ci, eci)) || (rc = up(&o->ell_m, em)) || (rc = up(&o->ell_s, es)))) return rc;
    {
        const std::vector<float> em32(em.begin(), em.end()), es32(es.begin(), es.end());
        const std::vector<float> dm32(dm.begin(), dm.end()), ds32(ds.begin(), ds.end());
        if (ell_w && ((rc = up(&o->ell_m32, em32)) || (rc = up(&o->ell_s32, es32)))) return rc;
        if ((rc = up(&o->dm32, dm32)) || (rc = up(&o->ds32, ds32))) return rc;
    }
    std::vector<int32_t> vd(n);
    for (int d = 0; d < g.n_dom; d++)
        for (int64_t v = dv0[d]; v < dv0[d + 1]; v++) vd[v] = d;
    if ((rc = up(&o->vdom, vd))) return rc;
    // Pade coefficients and, per domain, the damped wavenumber of its block
    // (Sec. 2.3): the domain's own k_d, or the exterior k0 for every block
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
    const int nd = g.n_dom;
    o->n_pade = N;
    o->C0 = make_double2(C0.real(), C0.imag());
    o->ikk.resize(nd);
    o->inv_keps2.resize(nd);
    o->A.resize((size_t)nd * N);
    o->B.resize((size_t)nd * N);
    std::vector<double2> pb((size_t)2 * nd), pc((size_t)2 * nd);
    for (int d = 0; d < nd; d++) {
        const cd kd = ctx->opts.osrc_wavenumber == 1 ? cd(ctx->k0re, ctx->k0im) : cd(ctx->doms[d].kre, ctx->doms[d].kim);
        const double eps = 0.4 * std::pow(kd.real(), ctx->opts.eps_exponent) * std::pow(reps, -2.0 / 3.0);
        const cd keps = kd + cd(0, eps);
        const cd ik2 = 1.0 / (keps * keps);
        const cd ik = cd(0, 1) * kd;
        o->ikk[d] = make_double2(ik.real(), ik.imag());
        o->inv_keps2[d] = make_double2(ik2.real(), ik2.imag());
        for (int l = 0; l < N; l++) {
            const cd den = 1.0 + bl[l] * (e - 1.0);
            const cd Al = std::exp(cd(0, -0.5 * th)) * al[l] / (den * den) * ik2;
            const cd Bl = e * bl[l] / den * ik2;
            o->A[(size_t)d * N + l] = make_double2(Al.real(), Al.imag());
            o->B[(size_t)d * N + l] = make_double2(Bl.real(), Bl.imag());
        }
        const cd inv = 1.0 / ik;
        pb[2 * d] = o->ikk[d];
        pb[2 * d + 1] = make_double2(1.0, 0.0);
        pc[2 * d] = make_double2(1.0, 0.0);
        pc[2 * d + 1] = make_double2(inv.real(), inv.imag());
    }
    if ((rc = up(&o->dA, o->A)) || (rc = up(&o->post_b, pb)) || (rc = up(&o->post_c, pc))) return rc;
    o->nblk = (int)std::min<int64_t>(128, (n + SP_THREADS - 1) / SP_THREADS);
    if ((rc = ensure_osrc_batch(ctx, o, 1))) return rc;
    o->tol = ctx->osrc_tol;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->osrc_ready = true;
    return BEM_OK;
}

// Solve (M - beta_s S) x_s = b_s for s < n_sys (b already in o->b, shifts
// in o->beta); solutions in o->x.  The iterations run in batches of
// GRAPH_ITERS as one captured CUDA graph (iteration parity is all the
// kernels take from the iteration count, so one graph serves every batch);
// convergence flags are read back between batches.
static void cocg_iteration_launches(OsrcState* o, CocgArgs a, int n_sys, cudaStream_t st) {
    const dim3 grid(o->nblk, n_sys);
    for (int k = 0; k < GRAPH_ITERS; k++) {
        a.it = k;
        cocg_spmv<<<grid, SP_THREADS, 0, st>>>(a);
        cocg_update<<<grid, SP_THREADS, 0, st>>>(a);
        cocg_direction<<<grid, SP_THREADS, 0, st>>>(a);
        cocg_check<<<(n_sys + 31) / 32, 32, 0, st>>>(o->scal, n_sys, a.tol2);
    }
}

// Domains of up to this many vertices are solved one CTA per (system,
// domain); larger ones by the grid-wide kernels below.
constexpr int64_t CTA_SOLVE_MAX_NV = 1 << 16;

static int cocg_solve_grid(bem_ctx* ctx, int n_sys);

// shifts > 1: the systems come in groups of `shifts` that share the right-hand
// side and differ only in the shift (the Pade systems of one bracket row).
static int cocg_solve(bem_ctx* ctx, int n_sys, int shifts = 1) {
    OsrcState* o = ctx->osrc;
    // the grid-wide kernels serve domains too large or rows too wide for the CTA solvers
    const int mode = ctx->opts.osrc_solver;
    const bool big = o->max_dom_nv > CTA_SOLVE_MAX_NV || o->ell_w == 0;
    if (mode == 2 || (mode == 0 && big)) return cocg_solve_grid(ctx, n_sys);
    // automatic: a cluster of CL CTAs per (system, domain).  Measured on the
    // 41k-triangle rib scene (n_pade 8, 10 % tolerance), per application to 1 /
    // 8 / 16 right-hand sides: clusters 6.4 / 27.3 / 49.6 ms, one CTA per
    // system 24.0 / 51.3 / 68.1 ms, grid-wide kernels 11.9 / 99.3 / 201 ms.
    // Small domains (under 4,096 vertices, fewer than two rows per thread of a
    // cluster's CTAs) go to one CTA per system once there are enough systems to
    // occupy the SMs: on an 8k-triangle rib scene (384 systems x domains) one
    // CTA took 0.95 ms where the clusters took 1.56 ms; with fewer systems than
    // SMs the clusters spread the work wider (the 1,280-triangle sphere's solve
    // took 0.13 s with clusters, 0.16 s with one CTA per system).
    const bool clustered = mode == 3 || mode == 4 ||
                           (mode == 0 && (o->max_dom_nv >= 4096 || (int64_t)n_sys * o->n_dom < 152));
    // the shifts of a group in one cluster (mode 4, or automatic once measured to pay)
    const bool grouped = clustered && (mode == 4 || (mode == 0 && SHIFT_GROUPS_AUTO)) && (shifts == 4 || shifts == 8) &&
                         n_sys % shifts == 0;
    CocgCtaArgs a{};
    a.n = o->n; a.eci = o->ell_ci; a.em = o->ell_m; a.es = o->ell_s; a.dm = o->dm; a.ds = o->ds;
    a.beta = o->beta; a.b = o->b; a.x = o->x; a.r = o->r; a.z = o->z; a.p = o->p; a.q = o->q;
    a.dom_v0 = o->dom_v0; a.n_dom = o->n_dom; a.tol2 = o->tol * o->tol; a.stat = o->stat;
    // a loose solve inside a flexible GMRES that has not converged by then is stagnating
    a.max_iter = ctx->osrc_strict ? o->max_iter : std::min(o->max_iter, 2000);
    const unsigned ctas = (unsigned)(n_sys * o->n_dom);
    CK(cudaMemsetAsync(o->stat, 0, 2 * sizeof(unsigned long long), ctx->stream));
    if ((mode == 1 || mode == 3 || mode == 4) && o->ell_w == 0)
        return ctx->fail(BEM_ERR_INVALID_ARG, "mesh rows too wide for the CTA solvers");
    // loose solves (inside a flexible GMRES) run in FP32: the same iteration on
    // FP32 vectors, with the same choice between clusters and single CTAs
    if (!ctx->osrc_strict && o->tol >= 1e-4 && !grouped && o->ell_w) {
        CocgArgs32 b{};
        b.n = o->n; b.eci = o->ell_ci; b.em = o->ell_m32; b.es = o->ell_s32; b.dm = o->dm32; b.ds = o->ds32;
        b.beta = o->beta; b.b = o->b; b.xout = o->x;
        b.x = o->x32; b.r = o->r32; b.z = o->z32; b.p = o->p32; b.q = o->q32;
        b.dom_v0 = o->dom_v0; b.n_dom = o->n_dom; b.tol2 = (float)(o->tol * o->tol); b.max_iter = a.max_iter;
        b.stat = o->stat;
        if (clustered) {
            const unsigned grid = ctas * CL;
            if (o->ell_w == 8) cocg_cluster32_kernel<256, 8><<<grid, 256, 0, ctx->stream>>>(b);
            else if (o->ell_w == 12) cocg_cluster32_kernel<256, 12><<<grid, 256, 0, ctx->stream>>>(b);
            else cocg_cluster32_kernel<256, 16><<<grid, 256, 0, ctx->stream>>>(b);
        } else if (ctas <= 152) {
            if (o->ell_w == 8) cocg_cta32_kernel<1024, 8><<<ctas, 1024, 0, ctx->stream>>>(b);
            else if (o->ell_w == 12) cocg_cta32_kernel<1024, 12><<<ctas, 1024, 0, ctx->stream>>>(b);
            else cocg_cta32_kernel<1024, 16><<<ctas, 1024, 0, ctx->stream>>>(b);
        } else {
            if (o->ell_w == 8) cocg_cta32_kernel<256, 8><<<ctas, 256, 0, ctx->stream>>>(b);
            else if (o->ell_w == 12) cocg_cta32_kernel<256, 12><<<ctas, 256, 0, ctx->stream>>>(b);
            else cocg_cta32_kernel<256, 16><<<ctas, 256, 0, ctx->stream>>>(b);
        }
        ctx->launches += 1;
        CK(cudaGetLastError());
        return BEM_OK;  // loose: the counters are not read back
    }
    // up to one wave: 1024 threads per CTA (one CTA per SM, shortest iterations);
    // beyond: 256 threads, three CTAs per SM
    if (grouped) {
        const unsigned grid = (unsigned)(n_sys / shifts * o->n_dom * CL);
        if (shifts == 8) {
            if (o->ell_w == 8) cocg_cluster_shift_kernel<256, 8, 8><<<grid, 256, 0, ctx->stream>>>(a);
            else if (o->ell_w == 12) cocg_cluster_shift_kernel<256, 12, 8><<<grid, 256, 0, ctx->stream>>>(a);
            else cocg_cluster_shift_kernel<256, 16, 8><<<grid, 256, 0, ctx->stream>>>(a);
        } else {
            if (o->ell_w == 8) cocg_cluster_shift_kernel<256, 8, 4><<<grid, 256, 0, ctx->stream>>>(a);
            else if (o->ell_w == 12) cocg_cluster_shift_kernel<256, 12, 4><<<grid, 256, 0, ctx->stream>>>(a);
            else cocg_cluster_shift_kernel<256, 16, 4><<<grid, 256, 0, ctx->stream>>>(a);
        }
    } else if (clustered) {
        const unsigned grid = ctas * CL;
        if (o->ell_w == 8) cocg_cluster_kernel<256, 8><<<grid, 256, 0, ctx->stream>>>(a);
        else if (o->ell_w == 12) cocg_cluster_kernel<256, 12><<<grid, 256, 0, ctx->stream>>>(a);
        else cocg_cluster_kernel<256, 16><<<grid, 256, 0, ctx->stream>>>(a);
    } else if (ctas <= 152) {
        if (o->ell_w == 8) cocg_cta_kernel<1024, 8><<<ctas, 1024, 0, ctx->stream>>>(a);
        else if (o->ell_w == 12) cocg_cta_kernel<1024, 12><<<ctas, 1024, 0, ctx->stream>>>(a);
        else cocg_cta_kernel<1024, 16><<<ctas, 1024, 0, ctx->stream>>>(a);
    } else {
        if (o->ell_w == 8) cocg_cta_kernel<256, 8><<<ctas, 256, 0, ctx->stream>>>(a);
        else if (o->ell_w == 12) cocg_cta_kernel<256, 12><<<ctas, 256, 0, ctx->stream>>>(a);
        else cocg_cta_kernel<256, 16><<<ctas, 256, 0, ctx->stream>>>(a);
    }
    ctx->launches += 1;
    CK(cudaGetLastError());
    // a strict solve must reach its tolerance: read the counters back; a loose
    // one (inside a flexible GMRES) keeps whatever iterate it has, so nothing
    // is read and the host does not wait for the GPU here
    if (!ctx->osrc_strict) return BEM_OK;
    unsigned long long st[2];
    CK(cudaMemcpyAsync(st, o->stat, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    o->iters_last += (long long)st[0];
    if (st[1]) return ctx->fail(BEM_ERR_NOT_CONVERGED, "OSRC inner COCG solve did not converge");
    return BEM_OK;
}

static int cocg_solve_grid(bem_ctx* ctx, int n_sys) {
    OsrcState* o = ctx->osrc;
    CocgArgs a{};
    a.n = o->n; a.rp = o->rp; a.ci = o->ci; a.vm = o->vm; a.vs = o->vs; a.dm = o->dm; a.ds = o->ds;
    a.beta = o->beta; a.x = o->x; a.r = o->r; a.z = o->z; a.p = o->p; a.q = o->q; a.b = o->b;
    a.vdom = o->vdom; a.nd = o->n_dom;
    a.part = o->part; a.scal = o->scal; a.nblk = o->nblk; a.tol2 = o->tol * o->tol;
    const dim3 grid(o->nblk, n_sys);
    cocg_init<<<grid, SP_THREADS, 0, ctx->stream>>>(a);
    cocg_init_scalars<<<n_sys, SP_THREADS, 0, ctx->stream>>>(a);
    ctx->launches += 2;
    // graph of GRAPH_ITERS iterations for this system count and tolerance
    cudaGraphExec_t exec = nullptr;
    for (auto& g : o->graphs)
        if (g.n_sys == n_sys && g.tol == o->tol && g.beta == o->beta) exec = g.exec;
    if (!exec) {
        if (!o->cap) CK(cudaStreamCreateWithFlags(&o->cap, cudaStreamNonBlocking));
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(o->cap, cudaStreamCaptureModeThreadLocal));
        cocg_iteration_launches(o, a, n_sys, o->cap);
        CK(cudaStreamEndCapture(o->cap, &graph));
        CK(cudaGraphInstantiate(&exec, graph, 0));
        CK(cudaGraphDestroy(graph));
        o->graphs.push_back({n_sys, o->tol, o->beta, exec});
    }
    std::vector<double> sc(8 * n_sys);
    int it = 0;
    const int max_iter = ctx->osrc_strict ? o->max_iter : std::min(o->max_iter, 2000);
    while (it < max_iter) {
        CK(cudaGraphLaunch(exec, ctx->stream));
        it += GRAPH_ITERS;
        ctx->launches += 4 * GRAPH_ITERS;
        CK(cudaMemcpyAsync(sc.data(), o->scal, sc.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        bool any = false;
        for (int s = 0; s < n_sys; s++) any |= sc[8 * s + 6] != 0.0;
        if (!any) break;
    }
    o->iters_last += it;
    if (ctx->osrc_strict)
        for (int s = 0; s < n_sys; s++)
            if (sc[8 * s + 6] != 0.0 || sc[8 * s + 7] != 0.0)
                return ctx->fail(BEM_ERR_NOT_CONVERGED, "OSRC inner COCG solve did not converge");
    return BEM_OK;
}

// Inner tolerance of the preconditioner's sparse solves (relative residual).
void set_osrc_tolerance(bem_ctx* ctx, double tol) {
    if (ctx->osrc) ctx->osrc->tol = tol;
    ctx->osrc_tol = tol;
}

// y = P x for Galerkin rows x (system order); both device vectors.
// With u = M^-1 row, the bracket's g = M u is the row itself, so the Pade
// solves take the rows directly: 2 N_pade + 2 sparse solves per application.
int bem_ctx::apply_prec(const double2* xin, double2* yout) { return apply_prec_batch(xin, yout, 1); }

// The same for R right-hand sides [R][N] at once: all R (2 N_pade) Pade
// systems in one batched COCG, then all 2 R closing systems in another.
int bem_ctx::apply_prec_batch(const double2* xin, double2* yout, int64_t R) {
    bem_ctx* const ctx = this;
    int rc = osrc_build(this);
    if (rc) return rc;
    OsrcState* o = osrc;
    if ((rc = ensure_osrc_batch(this, o, R))) return rc;
    const int64_t n = o->n;
    const unsigned nb = (unsigned)((n + SP_THREADS - 1) / SP_THREADS);
    const int L = o->n_pade;
    const int ns = (int)(2 * L * R);
    // rows in vertex order: g[rb][0] = row1, g[rb][1] = row2
    rows_to_vertex<<<dim3(nb, (unsigned)R), SP_THREADS, 0, stream>>>(n, dev.v_dof1, dev.v_dof2, xin, o->g);
    // Pade solves w_{rb,i,l} = (M - B_l S)^-1 row_i, systems ordered [rb][row][l],
    // the shift of system s on domain d at be[s][d]
    replicate_rows<<<dim3(nb, (unsigned)ns), SP_THREADS, 0, stream>>>(n, L, o->g, o->b);
    o->beta = o->beta_pade;  // (device tables built with the batch buffers: no host copy per application)
    if ((rc = cocg_solve(this, ns, L))) return rc;
    // brackets; row 1 scaled by i k (the DtN weak form)
    BracketArgs ba{};
    ba.n = n; ba.rp = o->rp; ba.ci = o->ci; ba.vs = o->vs; ba.g = o->g; ba.w = o->x; ba.L = L; ba.C0 = o->C0;
    ba.A = o->dA; ba.post = o->post_b; ba.vdom = o->vdom;
    ba.out = o->b;
    bracket_kernel<<<dim3(nb, 2, (unsigned)R), SP_THREADS, 0, stream>>>(ba);
    // out1 = M^-1 (i k bracket_1);  out2 = (M - S/k_eps^2)^-1 bracket_2, then / (i k)
    o->beta = o->beta_close;
    if ((rc = cocg_solve(this, (int)(2 * R)))) return rc;
    BracketArgs cp{};  // scaled copy (no Pade terms): u_row = post_row * x_row
    cp.n = n; cp.rp = o->rp; cp.ci = o->ci; cp.vs = o->vs; cp.g = o->x; cp.w = nullptr; cp.L = 0;
    cp.C0 = make_double2(1.0, 0.0);
    cp.post = o->post_c; cp.vdom = o->vdom;
    cp.out = o->u;
    bracket_kernel<<<dim3(nb, 2, (unsigned)R), SP_THREADS, 0, stream>>>(cp);
    vertex_to_rows<<<dim3(nb, (unsigned)R), SP_THREADS, 0, stream>>>(n, dev.v_dof1, dev.v_dof2, o->u, yout);
    launches += 5;
    CK(cudaGetLastError());
    return BEM_OK;
}

int bem_ctx::apply_prec_ahat(const double2* x, double2* y, int precision) {
    int rc = apply_ahat(x, dev.ys2, precision);
    if (rc) return rc;
    return apply_prec(dev.ys2, y);
}
