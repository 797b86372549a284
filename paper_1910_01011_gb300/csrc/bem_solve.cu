// bem_solve.cu -- incident fields and right-hand sides (paper Sec. 2.3 eq.
// Galerkin_disc_rhs1: b_r = <gamma^{j,+} p_inc, eta_r>), with the same
// regular rule as the operator.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "ctx.h"
#include "internal.h"

using namespace gbem;

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

namespace gbem {

struct PlaneWaveArgs {
    const double4* pg;   // (dx, dy, dz, w)
    const double4* tc;
    const int4* slot_v;
    const double* slot_n;
    double d[3];
    double2 amp, k0;
    int64_t n_slots;
    double lam[QP][3];
    double2* tri_out;
};

// Per slot: <p_inc, phi_k> and <dp_inc/dn, phi_k> on the triangle with the
// regular rule; p_inc = amp exp(i k0 d.x), dp/dn = i k0 (d.n) p_inc.
__global__ void plane_wave_kernel(PlaneWaveArgs a) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.n_slots) return;
    if (a.slot_v[s].x < 0) return;
    const double4 c = a.tc[s / TT];
    const double dn = a.d[0] * a.slot_n[3 * s] + a.d[1] * a.slot_n[3 * s + 1] + a.d[2] * a.slot_n[3 * s + 2];
    double r[3][2][2] = {};
    for (int q = 0; q < QP; q++) {
        const double4 g = a.pg[s * QP + q];
        const double x = c.x + g.x, y = c.y + g.y, z = c.z + g.z;
        const double ph = a.d[0] * x + a.d[1] * y + a.d[2] * z;
        // exp(i k0 ph) with complex k0
        double sn, cs;
        sincos(a.k0.x * ph, &sn, &cs);
        const double m = exp(-a.k0.y * ph);
        const double er = m * cs, ei = m * sn;
        const double pr = a.amp.x * er - a.amp.y * ei, pi = a.amp.x * ei + a.amp.y * er;
        // i k0 dn p
        const double kr = -a.k0.y * dn, ki = a.k0.x * dn;
        const double qr = kr * pr - ki * pi, qi = kr * pi + ki * pr;
        for (int k = 0; k < 3; k++) {
            const double wl = g.w * a.lam[q][k];
            r[k][0][0] += wl * pr;
            r[k][0][1] += wl * pi;
            r[k][1][0] += wl * qr;
            r[k][1][1] += wl * qi;
        }
    }
    for (int k = 0; k < 3; k++) {
        a.tri_out[(s * 3 + k) * 2] = make_double2(r[k][0][0], r[k][0][1]);
        a.tri_out[(s * 3 + k) * 2 + 1] = make_double2(r[k][1][0], r[k][1][1]);
    }
}

}  // namespace gbem

int bem_ctx::apply_prec(const double2*, double2*) {
    return fail(BEM_ERR_STATE, "the OSRC preconditioner is not available in this build");
}

int bem_ctx::apply_prec_ahat(const double2*, double2*, int) {
    return fail(BEM_ERR_STATE, "the OSRC preconditioner is not available in this build");
}

extern "C" {

int bem_set_plane_wave(bem_ctx* ctx, const double dir[3], bem_z amp) {
    if (!ctx || !dir) return BEM_ERR_INVALID_ARG;
    double n = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    if (!(n > 0)) return ctx->fail(BEM_ERR_INVALID_ARG, "zero plane-wave direction");
    for (int i = 0; i < 3; i++) ctx->pw_dir[i] = dir[i] / n;
    ctx->pw_amp[0] = amp.re;
    ctx->pw_amp[1] = amp.im;
    ctx->field_kind = 1;
    ctx->n_rhs = 1;
    ctx->rhs_ready = false;
    return BEM_OK;
}

int bem_set_transducer(bem_ctx* ctx, const double* c, const double* n, const double* r, int64_t n_elem,
                       double omega_rho0) {
    if (!ctx || !c || !n || !r || n_elem < 1) return BEM_ERR_INVALID_ARG;
    ctx->tr_c.assign(c, c + 3 * n_elem);
    ctx->tr_n.assign(n, n + 3 * n_elem);
    ctx->tr_r.assign(r, r + n_elem);
    ctx->omega_rho0 = omega_rho0;
    ctx->field_kind = 2;
    ctx->tr_w.assign(2 * n_elem, 0.0);
    for (int64_t m = 0; m < n_elem; m++) ctx->tr_w[2 * m] = 1.0;
    ctx->n_rhs = 1;
    ctx->rhs_ready = false;
    return BEM_OK;
}

int bem_set_excitations(bem_ctx* ctx, const bem_z* w, int64_t n_rhs) {
    if (!ctx || !w || n_rhs < 1) return BEM_ERR_INVALID_ARG;
    if (ctx->field_kind != 2) return ctx->fail(BEM_ERR_STATE, "set a transducer first");
    const int64_t ne = (int64_t)ctx->tr_r.size();
    ctx->tr_w.assign((const double*)w, (const double*)w + 2 * ne * n_rhs);
    ctx->n_rhs = n_rhs;
    ctx->rhs_ready = false;
    return BEM_OK;
}

int bem_rhs(bem_ctx* ctx, bem_z* b, int on_device) {
    if (!ctx || !b) return BEM_ERR_INVALID_ARG;
    CK(cudaSetDevice(ctx->device));
    int rc = ctx->finalize();
    if (rc) return rc;
    if (ctx->field_kind != 1) return ctx->fail(BEM_ERR_STATE, "no plane wave set (transducer right-hand sides are not available in this build)");
    const Geometry& g = ctx->geo;
    PlaneWaveArgs a{};
    a.pg = ctx->dev.pg64;
    a.tc = ctx->dev.tc;
    a.slot_v = ctx->dev.slot_v;
    a.slot_n = ctx->dev.slot_n;
    for (int i = 0; i < 3; i++) a.d[i] = ctx->pw_dir[i];
    a.amp = make_double2(ctx->pw_amp[0], ctx->pw_amp[1]);
    a.k0 = make_double2(ctx->k0re, ctx->k0im);
    a.n_slots = g.n_slots;
    for (int q = 0; q < QP; q++)
        for (int k = 0; k < 3; k++) a.lam[q][k] = ctx->quad.lam[q][k];
    a.tri_out = ctx->dev.tri_out;
    plane_wave_kernel<<<(unsigned)((g.n_slots + 127) / 128), 128, 0, ctx->stream>>>(a);
    CK(cudaGetLastError());
    ReduceArgs ra{};
    ra.vc_ptr = ctx->dev.vc_ptr; ra.vc_idx = ctx->dev.vc_idx; ra.v_dof1 = ctx->dev.v_dof1; ra.v_dof2 = ctx->dev.v_dof2;
    ra.tri_out = ctx->dev.tri_out; ra.v_begin = 0; ra.v_end = g.n_vert;
    ra.y = on_device ? (double2*)b : ctx->dev.ys;
    CK(launch_reduce(ra, ctx->stream));
    if (!on_device) {
        CK(cudaMemcpyAsync(b, ctx->dev.ys, g.n_dof * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return BEM_OK;
}

int bem_default_solve_opts(bem_solve_opts* o) {
    if (!o) return BEM_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof *o);
    o->restart = 100;
    o->max_iter = 2000;
    o->tol = 1e-8;
    o->precision = BEM_PREC_FP64;
    o->precondition = 1;
    o->inner_tol = 1e-4;
    o->max_refine = 10;
    return BEM_OK;
}

int bem_solve(bem_ctx* ctx, const bem_solve_opts*, bem_solve_report*) {
    if (!ctx) return BEM_ERR_INVALID_ARG;
    return ctx->fail(BEM_ERR_STATE, "bem_solve is not available in this build");
}

int bem_get_traces(bem_ctx* ctx, int32_t, int64_t, bem_z*, bem_z*, int) {
    if (!ctx) return BEM_ERR_INVALID_ARG;
    return ctx->fail(BEM_ERR_STATE, "no solve has run");
}

}  // extern "C"
