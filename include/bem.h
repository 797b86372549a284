/*
 * bem.h -- C ABI of the GB300 multiple-domain Galerkin BEM library
 * (Helmholtz transmission problem, PMCHWT multitrace formulation with the
 * OSRC block-diagonal preconditioner; arXiv 1910.01011).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns BEM_OK (0) or a negative BEM_ERR_* code; the
 *   message of the last failure is bem_last_error(ctx).  No C++ exception
 *   crosses this boundary.  A context is used by one host thread at a time.
 * - Complex numbers are interleaved (re, im) doubles: bem_z.
 * - Meshes: vertices double[nv][3], triangles int32[nt][3] ordered
 *   counter-clockwise seen from outside the domain, so that the right-hand
 *   normal points out of the domain (the normal n^j of the traces, paper
 *   Sec. 2.1 eq. traces).  Surfaces must be closed, conforming and
 *   orientable; different domains must not touch (no triple points,
 *   Sec. 2).  The library copies every input array; the caller keeps
 *   ownership of its buffers.
 * - System order of unknowns and rows (paper Sec. 2.2 eq.
 *   Form2_matrix_format_p2 with the column permutation of Sec. 2.3): per
 *   domain j, [psi_j (nv_j); phi_j (nv_j)] = [gamma_N^+ p_tot; gamma_D^+ p_tot]
 *   at the domain's vertices, domains concatenated in creation order.  Rows:
 *   per domain [row1 (the V row); row2 (the W row)].
 * - Device pointers (on_device = 1) must be device memory of the context's
 *   device; work is queued on the context's stream and the call returns
 *   without synchronising unless stated.  Host pointers (on_device = 0)
 *   make the call copy through the context's stream and synchronise.
 */
#ifndef GBEM_BEM_H
#define GBEM_BEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bem_ctx bem_ctx;
typedef struct {
    double re, im;
} bem_z;

enum {
    BEM_OK = 0,
    BEM_ERR_INVALID_ARG = -1,
    BEM_ERR_MESH_INVALID = -2,
    BEM_ERR_OUT_OF_BUDGET = -3,
    BEM_ERR_NOT_CONVERGED = -4,
    BEM_ERR_TIMEOUT = -5,
    BEM_ERR_CUDA = -6,
    BEM_ERR_STATE = -7
};

/* Arithmetic of an operator application. */
enum {
    BEM_PREC_FP64 = 0, /* FP64 everywhere (the baseline path) */
    BEM_PREC_FP32 = 1, /* FP32 far field with tile-local phase, FP64 near field and output */
    BEM_PREC_BF16X3 = 2, /* assembled complex64 A_hat (set-up once; N^2 x 12 bytes of BF16 planes kept)
                            applied to all right-hand sides at once by the split-BF16 tensor-core GEMM */
    BEM_PREC_FP64_ASSEMBLED = 3 /* assembled complex128 A_hat (set-up once in FP64; N^2 x 16 bytes kept),
                                   applied by a complex GEMM/GEMV: the fast FP64 residual */
};

/* Operators for bem_apply. */
enum {
    BEM_OP_AHAT = 0,     /* y = A_hat x, the PMCHWT Galerkin system (Sec. 2.2-2.3) */
    BEM_OP_PREC = 1,     /* y = P x, the OSRC preconditioner on Galerkin rows (Sec. 2.3) */
    BEM_OP_PREC_AHAT = 2 /* y = P A_hat x */
};

typedef struct {
    int32_t n_gauss_singular;  /* Gauss points per direction of the Sauter-Schwab rules (default 6) */
    int32_t chunk_tiles;       /* source tiles per far-field work item; 0 = automatic */
    int64_t hbm_budget_bytes;  /* device memory cap for this context; 0 = no cap */
    int32_t n_pade;            /* OSRC Pade terms (default 4; paper: 4 spheres, 8 anatomy, Sec. 3) */
    double pade_theta;         /* OSRC branch-cut rotation (default pi/3) */
    double r_eps;              /* OSRC damping radius R_eps (Sec. 2.3 eq. OSRC_DtN_NtD_maps); <= 0: 1/10 of the largest domain diameter */
    double eps_exponent;       /* exponent of k in eps = 0.4 k^e R_eps^(-2/3); default 1/3 */
    double osrc_tol;           /* relative residual of the preconditioner's sparse solves in bem_apply
                                  (default 1e-11); bem_solve sets its own (bem_solve_opts.prec_tol) */
    int32_t osrc_solver;       /* sparse solver of the preconditioner: 0 automatic (by the number of systems
                                  and the domain sizes), 1 one CTA per system and domain, 2 grid-wide
                                  kernels, 3 one 8-CTA thread-block cluster per system and domain, 4 as 3
                                  with the Pade shifts of one right-hand side in one cluster; same results
                                  within osrc_tol */
    int32_t osrc_wavenumber;   /* wavenumber each domain's OSRC block is built at (Sec. 2.3 eq. OSRC_prec_blocks
                                  writes the blocks with a "+" superscript and leaves this open): 0 (default)
                                  the domain's own k_j, 1 the exterior k0.  Only the GMRES iteration count
                                  depends on it; k_j needed 1.3-2.1x fewer iterations on every scene measured */
    int32_t fp64_far;          /* far field of the FP64 matrix-free operator: 0 (default) double-float arithmetic
                                  on the FP32 pipes (pairs of FP32 numbers, ~1e-13 relative, phases below
                                  ~100,000 rad), 1 native FP64 (GB300 runs FP64 at ~1/64 of the FP32 rate) */
} bem_opts;

/* Fill opts with the defaults above. */
int bem_default_opts(bem_opts* opts);

/* Create a context on CUDA device `device`, queueing all work on the CUDA
 * stream `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * opts may be NULL.  *out receives the context. */
int bem_create(bem_ctx** out, int device, void* cuda_stream, const bem_opts* opts);

/* Release the context and all device memory it owns.  NULL is a no-op. */
int bem_destroy(bem_ctx* ctx);

/* Exterior medium Omega^0: wavenumber k0 (Im >= 0) and density rho0
 * (Sec. 2.1 eq. model). */
int bem_set_exterior(bem_ctx* ctx, bem_z k0, double rho0);

/* Add a domain Omega^j with its closed surface, interior wavenumber k_j and
 * density rho_j.  *domain_id receives its index (0, 1, ...).  Returns
 * BEM_ERR_MESH_INVALID for out-of-range or degenerate triangles or an open
 * surface (an edge not shared by exactly two triangles). */
int bem_add_domain(bem_ctx* ctx, const double* verts, int64_t nv, const int32_t* tris, int64_t nt, bem_z k,
                   double rho, int32_t* domain_id);

/* Change the material of an existing domain (rebuilds the near field). */
int bem_set_material(bem_ctx* ctx, int32_t domain_id, bem_z k, double rho);

/* Number of unknowns N = sum_j 2 nv_j. */
int bem_num_dofs(const bem_ctx* ctx, int64_t* n);

/* Number of Green's-function evaluations of one far-field application of
 * A_hat (one per quadrature-point pair and wavenumber). */
int bem_interaction_count(const bem_ctx* ctx, int64_t* n);

/* y = op(x) for n_rhs right-hand sides stored one after another (x, y:
 * n_rhs * N complex each, system order).  precision: BEM_PREC_*.
 * x and y must not overlap. */
int bem_apply(bem_ctx* ctx, int op, const bem_z* x, bem_z* y, int64_t n_rhs, int precision, int on_device);

/* One Calderon block A_k^{ji} = [[-K, V], [W, K']] (App. A) between the
 * surfaces of test domain j and trial domain i at wavenumber k, in the
 * paper's order: x = [phi_i; psi_i] (2 nv_i), y = [row1; row2] (2 nv_j).
 * For i == j the touching pairs use the singular rules. */
int bem_apply_block(bem_ctx* ctx, int32_t test_domain, int32_t trial_domain, bem_z k, const bem_z* x, bem_z* y,
                    int precision, int on_device);

/* Allocation-free variant of bem_apply(BEM_OP_AHAT, BEM_PREC_FP32) for one
 * vector.  The paper has no counterpart: this exists for callers that
 * cannot let the library allocate device memory during the call, such as a
 * process whose device memory is reserved by another allocator or a
 * latency-critical loop that must not enter the CUDA allocator.
 * x, y: device pointers (N complex each, system order, must not overlap),
 * work queued on the context's stream, no synchronisation.
 * The context must already be prepared by an earlier allocating call
 * (bem_apply on it); otherwise BEM_ERR_STATE, and nothing is allocated.
 * The far-field scratch is a fixed 64 MiB array inside the library (held on
 * every GPU that loads the library until exit); target tiles are processed
 * in batches that fit it.  A problem whose single target tile needs more than
 * that scratch is rejected with BEM_ERR_OUT_OF_BUDGET.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  All calls
 * share the array: calls that overlap on the GPU (other streams or other
 * contexts on the same device) race on it and must be serialised by the
 * caller.  The scratch is fully rewritten by every call; nothing needs to be
 * cleared between calls.  The call does not synchronise, so a bounded wait
 * that timed out inside its kernels is not reported by it: the kernel sets
 * the context's device error flag, and the next call that checks the flag
 * (bem_apply with on_device = 0, bem_solve, bem_field) returns
 * BEM_ERR_TIMEOUT and clears it. */
int bem_apply_noalloc(bem_ctx* ctx, const bem_z* x, bem_z* y);

/* Dense complex product on the tensor cores: Y = A X with A (m x k),
 * X (n_rhs x k, each right-hand side contiguous) and Y (n_rhs x m), all
 * complex64 (interleaved float re, im) device arrays.  Split BF16 with FP32
 * accumulation (the GEMM of the assembled-operator path): each real part
 * split into three BF16 terms and the six products down to ~2^-24 kept.  Work and scratch use the context's stream and budget; the
 * call synchronises. */
int bem_zgemm_bf16x3(bem_ctx* ctx, int64_t m, int64_t k, int64_t n_rhs, const void* A, const void* X, void* Y);

/* Incident field: a plane wave amp * exp(i k0 d.x) (d normalised here). */
int bem_set_plane_wave(bem_ctx* ctx, const double dir[3], bem_z amp);

/* Incident field: n_elem flat pistons (centres, unit normals, radii: host
 * arrays) radiating by the Rayleigh integral with unit normal velocity,
 * p = -(i omega rho0 / 2 pi) sum_m w_m int exp(i k0 R)/R dS; omega_rho0 is
 * omega * rho0.  Piston weights come from bem_set_excitations. */
int bem_set_transducer(bem_ctx* ctx, const double* centres, const double* normals, const double* radii,
                       int64_t n_elem, double omega_rho0);

/* Piston weights of n_rhs excitations, w[r * n_elem + m] (host array). */
int bem_set_excitations(bem_ctx* ctx, const bem_z* w, int64_t n_rhs);

/* Right-hand side b = [<gamma_D p_inc, phi_r>; <gamma_N p_inc, phi_r>] per
 * domain (Sec. 2.3 eq. Galerkin_disc_rhs1) for every excitation (n_rhs * N
 * complex; one vector for a plane wave). */
int bem_rhs(bem_ctx* ctx, bem_z* b, int on_device);

typedef struct {
    int32_t restart;       /* GMRES restart (paper: 100, Sec. 3) */
    int32_t max_iter;      /* total inner iterations cap */
    double tol;            /* target relative residual of the returned traces */
    int32_t precision;     /* BEM_PREC_FP64: plain FP64 GMRES; BEM_PREC_FP32: FP32 inner, FP64 refinement */
    int32_t precondition;  /* 1 = OSRC preconditioner */
    double inner_tol;      /* inner relative tolerance of the mixed-precision path (default 1e-4; an inner
                              solve that only needs a smaller reduction to reach tol stops there) */
    int32_t max_refine;    /* outer refinement cap (default 10) */
    int32_t operator_mode; /* 0: matrix-free operators; 1: assembled operators (BF16-split tensor-core
                              GEMM inside GMRES, complex128 GEMV for FP64 residuals), set up once and
                              kept on the device for later solves; 2: automatic, assembled where those
                              operators take at most 4 GiB (36 N^2 bytes, N <= 10,922), else
                              matrix-free */
    int32_t batch_rhs;     /* >1: excitations are solved in blocks of up to batch_rhs right-hand sides,
                              R independent GMRES runs in lockstep (or one block GMRES, block_gmres) whose
                              operator and preconditioner applications act on all R columns at once (one
                              GEMM per application with operator_mode 1); each column stops on its own
                              residual.  0 or 1: one excitation after another (default).  The results do
                              not depend on it (within the tolerance). */
    int32_t flexible;      /* 1 (default): the preconditioner is applied on the right, u = P y, inside a
                              flexible GMRES that keeps the preconditioned basis, so its sparse solves may
                              stop at the loose tolerance prec_tol; GMRES then measures the residual of
                              A_hat itself.  0: the paper's left composition P A_hat u = P b with plain
                              GMRES (sparse solves to 1/100 of the GMRES tolerance).  Same solution. */
    double prec_tol;       /* relative residual of the preconditioner's sparse solves inside the solve;
                              0 = automatic (0.3 flexible, 1/100 of the GMRES tolerance otherwise) */
    int32_t block_gmres;   /* with batch_rhs > 1: 0 (default) R independent GMRES runs in lockstep; 1 block
                              GMRES, one Krylov space shared by the block's R columns and grown by R vectors per
                              step (restart then counts steps of R vectors; report.iterations counts steps per
                              column, each one application of the operator and preconditioner to R vectors);
                              blocks are at most 16 columns wide, a larger batch is split evenly.  Same
                              solution. */
    int32_t recycle;       /* batched solves (batch_rhs > 1): keep up to this many solved pairs (b, u) of the
                              context (orthonormalised: Q, U' with A U' = Q) and start every later solve of the
                              same operator from u0 = U' Q^H b, so only the part of b outside the span of the
                              earlier right-hand sides is left to GMRES (with as many pairs as pistons, any
                              excitation of that transducer starts converged).  0 (default): off.  Kept across
                              bem_set_transducer and bem_set_excitations; dropped when the operator changes
                              (bem_set_exterior, bem_set_material).  Same solution. */
} bem_solve_opts;

typedef struct {
    int32_t iterations;    /* total inner GMRES iterations */
    int32_t refinements;   /* outer FP64 refinement steps */
    double residual;       /* final FP64 relative residual ||b - A_hat u|| / ||b|| */
    double seconds;        /* wall time of the solve */
} bem_solve_report;

int bem_default_solve_opts(bem_solve_opts* o);

/* Solve A_hat u = b for every excitation set by bem_set_plane_wave /
 * bem_set_excitations.  Returns BEM_ERR_NOT_CONVERGED (report filled,
 * traces kept) when the tolerance is not met. */
int bem_solve(bem_ctx* ctx, const bem_solve_opts* opts, bem_solve_report* report);

/* Traces of the last solve for excitation `rhs` on domain j:
 * dirichlet = gamma_D p_tot, neumann = gamma_N^+ p_tot (exterior side;
 * the interior Neumann trace is rho_j/rho_0 times it, eq. Form1_BCs). */
int bem_get_traces(bem_ctx* ctx, int32_t domain_id, int64_t rhs, bem_z* dirichlet, bem_z* neumann, int on_device);

/* Excitation superposition (no counterpart as an entry point in the paper;
 * it follows from the linearity of eq. Galerkin_disc_rhs1 in the piston
 * weights).  bem_solve_basis solves every piston of the transducer alone
 * (n_elem unit excitations, with the given solve options; use batch_rhs) and
 * keeps the n_elem solutions on the device; the caller's excitations set by
 * bem_set_excitations are left as they were.  bem_superpose then returns the
 * solutions for any weights w [n_exc][n_elem] (complex, host or device) as
 * u = w x basis, [n_exc][bem_num_dofs], in the system order of
 * bem_get_solution, with one complex GEMM.  The residual of a superposed
 * solution is bounded by the basis tolerance times sum |w_m| ||b_m|| /
 * ||sum w_m b_m||, which for random phases grows like sqrt(n_elem): solve the
 * basis that much tighter.  STATE if no basis exists for the current
 * transducer; changing the mesh, materials or transducer drops it. */
int bem_solve_basis(bem_ctx* ctx, const bem_solve_opts* opts, bem_solve_report* report);
int bem_superpose(bem_ctx* ctx, const bem_z* w, int64_t n_exc, bem_z* u, int on_device);

/* The whole solution vector of excitation `rhs` of the last solve, in system
 * order: per domain j, [gamma_N^+ p_tot (n_v,j); gamma_D p_tot (n_v,j)]
 * (the unknown [psi; phi] of Sec. 2.3 after the column permutation).
 * u: bem_num_dofs complex values, host or device (on_device = 1). */
int bem_get_solution(bem_ctx* ctx, int64_t rhs, bem_z* u, int on_device);

/* Kernel timing for measurement: when enabled, the library records CUDA
 * events on its stream around every far-field kernel launch.
 * bem_profile_read synchronises the stream and returns the summed far-field
 * kernel time (ms), the number of far-field launches and the number of
 * kernels the library launched since the last reset (reset = 1 clears). */
int bem_profile_enable(bem_ctx* ctx, int enable);
int bem_profile_read(bem_ctx* ctx, double* far_ms, int64_t* far_launches, int64_t* kernel_launches, int reset);

/* Device memory of the context: bytes held now and the most it has held. */
int bem_memory_info(const bem_ctx* ctx, int64_t* used_bytes, int64_t* peak_bytes);

/* Upper estimate of the device bytes a solve of n_exc excitations with
 * options opts (null: defaults) needs at its peak, from the mesh sizes and
 * options alone (no device work): geometry, near-field blocks and their
 * build scratch, far-field partials, right-hand sides, GMRES basis, the
 * preconditioner's batched vectors and, with operator_mode 1, the assembled
 * operators. */
int bem_estimate_solve_bytes(const bem_ctx* ctx, int64_t n_exc, const bem_solve_opts* opts, int64_t* bytes);

/* Several meshes at once (no counterpart in the paper; for many small
 * problems, e.g. requests on small meshes, whose single applications leave
 * most SMs idle): y[i] = A_hat_i x[i] for the n contexts ctxs[i], FP32 far
 * field, every mesh's far-field work in ONE launch (work items of all meshes,
 * heaviest first), gathers, projections and reductions around it.  x[i], y[i]
 * are device vectors of ctxs[i]'s size.  The whole launch sequence is captured
 * into a CUDA graph owned by ctxs[0] and replayed on ctxs[0]'s stream while
 * the same contexts, vectors and device buffers are used; any change (another
 * vector, a context that reallocated, a different member list) captures anew.
 * The other contexts' pending work on their own streams is waited for first.
 * The source chunks are sized for the whole group (small meshes get long
 * chunks), so results match separate bem_apply calls at BEM_PREC_FP32 to FP32
 * rounding (a different summation order), not bit for bit.
 * Errors: INVALID_ARG (null pointers, repeated context, mixed devices). */
int bem_apply_group(bem_ctx* const* ctxs, int32_t n, const bem_z* const* x, bem_z* const* y);

/* Autotuner for the far-field launch shape (no counterpart in the paper):
 * times the whole operator application for source-chunk lengths 8..256
 * tiles and the built-in heuristic, keeps the fastest in the context
 * (bem_opts.chunk_tiles) and in a per-process cache keyed by the tile count,
 * number of domains and lossiness (a cached answer is reused without timing
 * unless best_ms is requested).  The results do not depend on the choice
 * beyond rounding order.  chunk_tiles / best_ms may be null. */
int bem_autotune(bem_ctx* ctx, int precision, int32_t* chunk_tiles, double* best_ms);

/* Total pressure at n_points points from the traces of excitation `rhs`
 * of the last solve, by the representation formula (App. A eq.
 * rep_formula_gen): for domain_of_point[i] = -1 (exterior)
 * p_inc + DL_k0(gamma_D p) - SL_k0(gamma_N p) over all surfaces; for
 * domain_of_point[i] = j, SL_kj((rho_j/rho_0) gamma_N p) - DL_kj(gamma_D p)
 * over domain j.  points: [n][3] doubles, out: n complex.  The caller says
 * which domain holds each point.  Accuracy degrades within about one element
 * size of a surface (regular rule).  Domain ids outside [-1, number of
 * domains) give BEM_ERR_INVALID_ARG: checked on the host for host arrays, by
 * the kernels for device arrays (those points are skipped and written as NaN). */
int bem_field(bem_ctx* ctx, int64_t rhs, const double* points, const int32_t* domain_of_point, int64_t n_points,
              bem_z* out, int on_device);

/* Arithmetic-rate probe for roofline denominators (no counterpart in the
 * paper): runs independent dependency chains of one operation on every SM of
 * the current device, on cuda_stream (a cudaStream_t, NULL = legacy default
 * stream), and returns the measured rate of one timed launch after a
 * warm-up.  which = 0: packed FP32 FMA (flops/s, FMA = 2 flops); 1: MUFU
 * sine (operations/s); 2: FP64 FMA (flops/s).  iters scales the work (each of
 * 16 x SMs x 256 threads issues iters x 128 operations).  Allocates and frees
 * 4 bytes of device memory.  Errors: INVALID_ARG, CUDA. */
int bem_peak_probe(int which, int iters, void* cuda_stream, double* ops_per_s);

/* Message of the last error on ctx (never NULL). */
const char* bem_last_error(const bem_ctx* ctx);

/* Host-only: the library's own quadrature tables, for comparison with an
 * independent derivation.  which = 0: regular triangle rule (rows l1, l2, w;
 * point P0 + l1 (P1-P0) + l2 (P2-P0), weights sum to 1); which = 1:
 * Gauss-Legendre on [0,1] with n points (rows node, weight).  *n_out
 * receives the number of rows; buf holds 3 * 64 doubles at least. */
int bem_quadrature_table(int which, int n, double* buf, int* n_out);

/* ---------------------------------------------------------------- serving
 *
 * A request loop for planning solves (no counterpart in the paper, which
 * solves one scene at a time).  A scene is a context with its meshes,
 * materials and transducer set (bem_set_transducer); the server takes it over
 * and keeps its device state (geometry, near-field corrections,
 * preconditioner, assembled operators) resident between requests.  A request
 * is a set of n_exc piston excitations (weights [n_exc][n_elem] complex) for
 * one scene.  Requests wait in a FIFO queue and start as soon as one of
 * `slots` workers and enough of the device-memory budget are free; queued
 * requests of the scene a worker picks are merged into one solve of up to
 * max_batch_rhs excitations (bem_solve with batch_rhs), and different scenes
 * run concurrently on their own streams.  Every device allocation of every
 * scene draws on one counter limited by hbm_budget_bytes; admission reserves
 * a solve's estimated need and evicts idle scenes, least recently used
 * first.  All calls are thread-safe.  Results are the solution vectors of
 * bem_get_solution, one per excitation, and do not depend on which other
 * requests shared the batch (within the solve tolerance). */
typedef struct bem_server bem_server;

enum { BEM_REQ_QUEUED = 0, BEM_REQ_RUNNING = 1, BEM_REQ_DONE = 2, BEM_REQ_FAILED = 3 };

typedef struct {
    int32_t slots;            /* concurrent solves (worker threads; default 2) */
    int32_t max_batch_rhs;    /* excitations merged into one solve (default 64) */
    int64_t hbm_budget_bytes; /* device bytes all scenes may hold together (default 150 GiB; 0 = no limit) */
    bem_solve_opts solve;     /* options of every solve (default: mixed precision, batch_rhs = max_batch_rhs,
                                 block_gmres = 1, operator_mode = 2, recycle = 256) */
    int32_t join;             /* 1 (default): requests for a scene whose mixed-precision solve is running join
                                 it at its next refinement boundary while the block (16 excitations with block
                                 GMRES, else batch_rhs) has room and the budget holds the growth of the solve's
                                 memory estimate.  0: they wait for the running solve to finish */
} bem_server_opts;

typedef struct {
    int64_t completed;        /* requests finished successfully */
    int64_t excitations;      /* excitations of those requests */
    int64_t failed;
    int64_t queued;
    int64_t running;          /* solves on the GPU now */
    int64_t batches;          /* solves run */
    double mean_batch_exc;    /* excitations per solve */
    double p50_ms, p99_ms, max_ms;  /* request latency, submit to result */
    double p50_wait_ms;       /* submit to start */
    double requests_per_s;    /* completed requests / (last completion - first submit) */
    double excitations_per_s;
    int64_t device_bytes;     /* held by all scenes now */
    int64_t peak_device_bytes;
    int64_t evictions;
    int64_t joined;           /* requests that joined a solve already running */
} bem_server_stats;

int bem_server_default_opts(bem_server_opts* opts);
/* Starts the workers.  Errors: INVALID_ARG (bad options), CUDA (no device). */
int bem_server_create(bem_server** out, int device, const bem_server_opts* opts);
/* Stops the workers after their current solves and destroys every scene. */
int bem_server_destroy(bem_server* server);
/* Takes ownership of ctx (the caller must neither use nor destroy it
 * afterwards); its device memory counts against the budget from now on.
 * STATE if ctx has no transducer or no domain. */
int bem_server_add_scene(bem_server* server, bem_ctx* ctx, int32_t* scene_id);
/* Sizes of a scene: solution length, pistons, device bytes held now. */
int bem_server_scene_info(bem_server* server, int32_t scene_id, int64_t* n_dofs, int64_t* n_elem,
                          int64_t* device_bytes);
/* Device bytes the server reserves for a solve of n_exc excitations of a
 * scene (its admission estimate, from the mesh sizes and solve options). */
int bem_server_estimate(bem_server* server, int32_t scene_id, int64_t n_exc, int64_t* bytes);
/* Queues a request; weights are copied.  Returns a handle at once. */
int bem_server_submit(bem_server* server, int32_t scene_id, const bem_z* weights, int64_t n_exc, int64_t* handle);
int bem_server_poll(bem_server* server, int64_t handle, int32_t* state);
/* Blocks until the request is done or failed (timeout_s < 0: no limit);
 * TIMEOUT if it is still queued or running when the time is up. */
int bem_server_wait(bem_server* server, int64_t handle, double timeout_s, int32_t* state);
/* Result of a finished request: u [n_exc][n_dofs] (host, may be null), the
 * solve report of its batch, its latency and the batch's excitation count.
 * Returns the request's own status (OK, NOT_CONVERGED with u filled,
 * OUT_OF_BUDGET, ...); STATE if it has not finished.  release = 1 forgets the
 * request afterwards. */
int bem_server_result(bem_server* server, int64_t handle, bem_z* u, bem_solve_report* report, double* latency_ms,
                      int64_t* batch_exc, int release);
int bem_server_get_stats(bem_server* server, bem_server_stats* stats);
/* Error text of a failed request ("" if it did not fail); valid until the
 * request is released. */
const char* bem_server_error(bem_server* server, int64_t handle);

#ifdef __cplusplus
}
#endif
#endif
