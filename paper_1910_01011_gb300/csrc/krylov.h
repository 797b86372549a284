// krylov.h -- FP64 device GMRES used by bem_solve.
#pragma once

#include <complex>
#include <functional>

#include "ctx.h"

namespace gbem {

struct Krylov {
    int64_t n = 0;
    int m = 0;
    double2 *V = nullptr, *w = nullptr, *t = nullptr, *part = nullptr, *h = nullptr, *y = nullptr;

    int ensure(bem_ctx* ctx, int64_t n, int m);
    void release(bem_ctx* ctx);
    int dot(bem_ctx* ctx, const double2* a, const double2* b, std::complex<double>* out);
    int norm(bem_ctx* ctx, const double2* a, double* out);
    int axpby(bem_ctx* ctx, std::complex<double> a, const double2* x, std::complex<double> b, const double2* z,
              double2* out);
    int gmres(bem_ctx* ctx, const std::function<int(const double2*, double2*)>& op, const double2* b, double2* x,
              int restart, double tol, int max_iter, int* iters, double* relres, bool zero_guess);
};

}  // namespace gbem
