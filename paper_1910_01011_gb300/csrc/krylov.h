// krylov.h -- FP64 device GMRES used by bem_solve.
#pragma once

#include <complex>
#include <functional>

#include "ctx.h"

namespace gbem {

struct Krylov {
    int64_t n = 0;
    int m = 0;
    int64_t R = 0;  // columns the buffers hold (batched GMRES)
    double2 *V = nullptr, *w = nullptr, *t = nullptr, *part = nullptr, *h = nullptr, *y = nullptr;
    double2* Z = nullptr;  // preconditioned basis of flexible GMRES, [m][R][n] (allocated on first use)
    double* sc = nullptr;
    // least-squares state of every column on the device (Givens rotations applied there)
    double2 *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr;  // [R][(m+1) m], [R][m], [R][m], [R][m+1]
    double *bn = nullptr, *res = nullptr;                               // [R] |b|, |residual| / |b|
    int *run = nullptr, *jr = nullptr, *its = nullptr;                  // [R]
    int* n_run = nullptr;                                               // [POLL] running-column counts
    int* n_run_host = nullptr;                                          // pinned copy of n_run
    cudaEvent_t poll_ev[4] = {nullptr, nullptr, nullptr, nullptr};

    Krylov() = default;
    Krylov(const Krylov&) = delete;
    Krylov& operator=(const Krylov&) = delete;
    ~Krylov() {  // device buffers belong to the context's allocations; the host-side poll objects are ours
        if (n_run_host) cudaFreeHost(n_run_host);
        if (hpin) cudaFreeHost(hpin);
        if (hs_pin) cudaFreeHost(hs_pin);
        for (auto& e : poll_ev)
            if (e) cudaEventDestroy(e);
    }

    int ensure(bem_ctx* ctx, int64_t n, int m, int64_t R = 1);
    void release(bem_ctx* ctx);
    int dot(bem_ctx* ctx, const double2* a, const double2* b, std::complex<double>* out);
    int norm(bem_ctx* ctx, const double2* a, double* out);
    // out = a x + b z over len entries (default n)
    int axpby(bem_ctx* ctx, std::complex<double> a, const double2* x, std::complex<double> b, const double2* z,
              double2* out, int64_t len = -1);
    // Solve op(x) = b.  With prec (flexible GMRES, right preconditioning):
    // z_j = prec(v_j), the basis grows with op(z_j) and x += Z y, so prec
    // may change from one application to the next (e.g. inner solves run to
    // a loose tolerance); residuals are those of op itself.
    using Op = std::function<int(const double2*, double2*)>;
    int gmres(bem_ctx* ctx, const Op& op, const double2* b, double2* x, int restart, double tol, int max_iter,
              int* iters, double* relres, bool zero_guess, const Op* prec = nullptr);
    int ensure_flexible(bem_ctx* ctx);
    // column norms of R vectors [R][n] (host out[R])
    int norms(bem_ctx* ctx, const double2* a, int64_t R, double* out);
    // R independent GMRES runs in lockstep: op maps [R][n] to [R][n] column
    // by column; column r stops once its own residual meets tol.
    int gmres_batch(bem_ctx* ctx, const Op& op, const double2* B, double2* X, int64_t R, int restart, double tol,
                    int max_iter, int* iters, double* relres, bool zero_guess, const Op* prec = nullptr);
    // Block GMRES over the R columns: one Krylov space shared by all columns,
    // grown by R vectors per step (op and prec applied to the R newest basis
    // vectors at once), restarted after `restart` steps; flexible (right
    // preconditioned) when prec is given.  iters[r] counts the steps.
    // fp32_basis: the basis is kept and orthogonalised in FP32 (an inner solve
    // of the mixed path, whose tolerance needs no FP64 orthogonalisation); the
    // vectors handed to op and prec and the solution update stay FP64.
    // deficient (optional): set when the block of starting residuals has
    // dependent columns (e.g. more excitations than pistons, or a zero one),
    // so that not one step could be taken; X is then as on entry (zero with
    // zero_guess) and the caller solves the columns another way.
    int gmres_block(bem_ctx* ctx, const Op& op, const double2* B, double2* X, int64_t R, int restart, double tol,
                    int max_iter, int* iters, double* relres, bool zero_guess, const Op* prec = nullptr,
                    bool fp32_basis = false, bool* deficient = nullptr);
    double2 *bpart = nullptr, *bC = nullptr;  // block GMRES scratch (allocated on first use)
    size_t bpart_n = 0, bC_n = 0;
    float2* b32 = nullptr;                    // FP32 basis and work blocks of the block GMRES
    size_t b32_n = 0;
    double2* hpin = nullptr;                  // pinned Hessenberg coefficients of two consecutive steps
    size_t hpin_n = 0;
    double2* hs_pin = nullptr;                // rotated block Hessenberg matrix (pinned host copy)
    double2 *hs_dev = nullptr, *gs_dev = nullptr;  // its device mirror; back-substitution right-hand sides
    size_t hs_n = 0;
    static void dfree_buf(bem_ctx* ctx, void** p);
};

}  // namespace gbem
