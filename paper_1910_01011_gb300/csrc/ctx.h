// ctx.h -- the opaque bem_ctx behind the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <functional>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

namespace gbem {

struct DeviceGeom {
    float4 *pg32 = nullptr, *pgp32 = nullptr, *tg32 = nullptr;  // pgp32: pg32 pair-interleaved
    double4 *pg64 = nullptr, *tg64 = nullptr, *tc = nullptr;
    int *tdom = nullptr, *tntri = nullptr;
    int2* dom_tiles = nullptr;
    int4* slot_v = nullptr;
    double *slot_P = nullptr, *slot_n = nullptr, *slot_area = nullptr, *slot_curl = nullptr, *pt_w = nullptr;
    int64_t* vc_ptr = nullptr;
    int32_t* vc_idx = nullptr;
    int64_t *v_dof1 = nullptr, *v_dof2 = nullptr;
    int64_t* np_ptr = nullptr;
    int32_t *np_src = nullptr, *np_code = nullptr, *np_tgt = nullptr;
    double* ss_tab[4] = {nullptr, nullptr, nullptr, nullptr};
    float* ss_tabf[4] = {nullptr, nullptr, nullptr, nullptr};  // the same as (hi [5 n], lo [5 n]) floats
    // working buffers
    float4 *pd32 = nullptr, *tcurl32 = nullptr;
    double4 *pd64 = nullptr, *tcurl64 = nullptr;
    double2* tri_out = nullptr;
    double2* kdom = nullptr;
    SlotCoef* coef = nullptr;
    int* err = nullptr;
    double2 *xs = nullptr, *ys = nullptr, *ys2 = nullptr;  // staging vectors (system size)
};

struct NearSet {
    int64_t n_pairs = 0;
    double2* nb64 = nullptr;
    float2* nb32 = nullptr;
};

struct BlockCache {
    int dom = -1;
    double kre = 0, kim = 0;
    SlotCoef* coef = nullptr;
    NearSet near;
};

struct ApplyMode {
    int tgt_dom_lo = 0, tgt_dom_hi = 0, src_dom_lo = 0, src_dom_hi = 0;
    double kre = 0, kim = 0;
    int slot1 = 0;
    const SlotCoef* coef = nullptr;
    const NearSet* near = nullptr;
};

// Launch arguments of one operator application (gather, far field, projection, reduction).
struct ApplyPlan {
    GatherArgs ga{};
    FarArgs32 fa32{};
    FarArgs64 fa64{};
    ProjectArgs pa{};
    ReduceArgs ra{};
    bool fp64 = false;
    int n_tgt = 0, n_chunks = 0;
};

// Several meshes applied together (bem_apply_group): the launch sequence,
// captured once as a CUDA graph and replayed while nothing it points to moved.
struct GroupCache {
    std::vector<bem_ctx*> ctxs;
    std::vector<uint64_t> gens;      // each context's allocation generation when captured
    std::vector<const void*> io;     // x and y pointers
    FarArgs32* table = nullptr;      // device [n] (owned by the first context)
    int4* work = nullptr;            // device [n_work]
    int64_t n_work = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
};

struct OsrcState;  // k_osrc.cu
struct SolveState; // bem_solve.cu

}  // namespace gbem

struct bem_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bem_opts opts{};
    std::string err;
    double k0re = 1.0, k0im = 0.0, rho0 = 1.0;
    std::vector<gbem::HostDomain> doms;
    // device state
    bool ready = false, near_ready = false, osrc_ready = false, rhs_ready = false;
    gbem::Quadrature quad;
    gbem::Geometry geo;
    gbem::DeviceGeom dev;
    gbem::NearSet pmchwt_near;
    std::vector<gbem::BlockCache> block_cache;
    void* partial = nullptr;
    size_t partial_bytes = 0;
    void* field_buf = nullptr;  // bem_field scratch (grow-only)
    size_t field_buf_bytes = 0;
    // far-field work list (heaviest (target tile, chunk) first) and the launch it was built for
    int2* far_work = nullptr;
    int far_work_key[6] = {-1, -1, -1, -1, -1, -1};
    // several right-hand sides in one far-field launch: densities, partials and the work list
    void* multi_buf = nullptr;
    size_t multi_buf_bytes = 0;
    void* multi64_buf = nullptr;  // FP64 multi-vector far field: densities, curls, partial potentials
    size_t multi64_buf_bytes = 0;
    struct DfGeom {                // double-float far field: split geometry, tables, constants
        bool ready = false;
        void* buf = nullptr;
        float4 *pgh = nullptr, *pgl = nullptr, *tgh = nullptr, *tgl = nullptr, *tch = nullptr, *tcl = nullptr;
        float4 *sctab = nullptr, *kdf = nullptr;
        float2* extab = nullptr;
        gbem::DfConsts c{};
    } dfg;
    void* dfv_buf = nullptr;       // double-float densities and curls of the vectors of one call
    size_t dfv_bytes = 0;
    // set by a request loop around bem_solve: at a refinement boundary of a
    // single-batch mixed solve, hands over up to `room` more excitations
    // (their weights appended to w, [k][n_elem] complex) and returns k
    std::function<int64_t(int64_t room, std::vector<double>& w)> join_hook;
    int4* multi_work = nullptr;
    int64_t multi_n_work = 0;
    int multi_key[3] = {-1, -1, -1};  // (n_chunks, chunk_tiles, groups) the list was built for
    std::vector<std::pair<void*, size_t>> allocs;
    size_t used_bytes = 0;
    size_t peak_bytes = 0;                     // largest used_bytes seen
    uint64_t gen = 0;                          // bumped by every device allocation and release
    gbem::GroupCache* group = nullptr;         // bem_apply_group state when this context leads a group
    std::atomic<int64_t>* pool = nullptr;      // shared device-memory counter (serving), or null
    int64_t pool_limit = 0;                    // limit of the shared counter (0: none)
    bool own_stream = false;                   // stream created by the library, destroyed with the context
    long long launches = 0;
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> far_events;
    double far_ms_acc = 0;
    long long far_count = 0;
    // assembled operator (split-BF16 planes) for BEM_PREC_BF16X3
    bool asm_ready = false;
    __nv_bfloat16* asm_planes = nullptr;
    int64_t asm_mpad = 0, asm_kpad = 0;
    void* asm_work = nullptr;
    size_t asm_work_bytes = 0;
    // assembled operator for FP64 refinement residuals: complex128 entries stored as
    // scaled FP32 (hi, lo) pairs, 16 bytes each (k_df64.cu)
    bool asm64_ready = false;
    double2* asm64 = nullptr;
    int* df_exp = nullptr;          // device [2]: exponents of asm64 and of the superposition basis
    void* df_work = nullptr;        // split vectors of the FP64-accurate products (grow-only)
    size_t df_work_bytes = 0;
    gbem::OsrcState* osrc = nullptr;
    double osrc_tol = 1e-11;  // relative residual of the preconditioner's sparse solves
    bool osrc_strict = true;  // a sparse solve that stops short of osrc_tol is an error (false: keep its iterate)
    gbem::SolveState* solve = nullptr;
    // incident field
    int field_kind = 0;  // 0 none, 1 plane wave, 2 transducer
    double pw_dir[3] = {0, 0, 1};
    double pw_amp[2] = {1, 0};
    std::vector<double> tr_c, tr_n, tr_r;
    double omega_rho0 = 0;
    std::vector<double> tr_w;  // n_rhs * n_elem * 2
    int64_t n_rhs = 1;

    int fail(int code, const std::string& msg);
    void* dalloc(size_t bytes, int* rc);
    void dfree(void* p);
    int finalize();
    int upload_materials();
    int build_near(gbem::NearSet& ns, int n_slot_k, double kre, double kim, const gbem::SlotCoef* coef_dev);
    int ensure_near();
    int ensure_partial(int n_chunks, bool fp64);
    int ensure_far_work(int tgt_b, int tgt_e, int src_b, int src_e, int chunk_tiles, int n_chunks, int slot1);
    void chunking(int n_tgt, int n_src, int* n_chunks, int* chunk_tiles) const;
    int plan_apply(const double2* x, double2* y, int precision, const gbem::ApplyMode& m, gbem::ApplyPlan& P,
                   int fill_tiles = 0);
    int run_apply(const double2* x, double2* y, int precision, const gbem::ApplyMode& m);
    int apply_ahat(const double2* x, double2* y, int precision);
    int apply_ahat_multi(const double2* x, double2* y, int64_t n_rhs);
    int apply_ahat64_multi(const double2* x, double2* y, int64_t n_rhs);
    int ensure_fardf();
    double df_extent(bool with_transducer) const;
    int check_df_phase(double kre, bool with_transducer);
    int far_df(const double4* pd, const double4* cu, int64_t R, int tgt_b, int tgt_e, int src_b, int src_e,
               int chunk_tiles, int n_chunks, int slot1, double kre, double kim, double* partial, int64_t rstride);
    int apply_prec(const double2* x, double2* y);
    int apply_prec_batch(const double2* x, double2* y, int64_t n_rhs);
    int apply_prec_ahat(const double2* x, double2* y, int precision);
    int check_device_error();
    int ensure_assembled();
    int apply_assembled(const double2* x, double2* y, int64_t n_rhs);
    int ensure_assembled64();
    int apply_assembled64(const double2* x, double2* y, int64_t n_rhs);
};

namespace gbem {
// Source chunks of the several-right-hand-side far field (bem_capi.cu): enough
// work items to fill the GPU, at most CHUNK_MAX tiles, and the partial
// potentials of all R vectors within 2 GiB where possible.
void multi_chunking(int n_tiles, int64_t n_pts, int64_t R, int* n_chunks, int* chunk_tiles);
void multi64_chunking(int n_tiles, int64_t R, int* n_chunks, int* chunk_tiles);
// excitations per batched solve: batch_rhs (at most n_exc), or for block GMRES
// the batch split evenly into blocks of at most 16 columns
int64_t solve_batch_width(const bem_solve_opts& o, int64_t n_exc);
// operator_mode 2 (automatic) resolved for n_dof unknowns: 1 (assembled) where
// the assembled operators take at most 4 GiB, else 0 (matrix-free)
inline int resolved_operator_mode(int mode, int64_t n_dof) {
    return mode != 2 ? mode : (36.0 * (double)n_dof * (double)n_dof <= 4.0 * 1073741824.0 ? 1 : 0);
}
// FP64-accurate complex products in FP32 arithmetic (k_df64.cu).
int df_prepare_inplace(bem_ctx* ctx, double2* v, int64_t n, int* e);
int df_gemv(bem_ctx* ctx, const float4* A, const int* eA, int64_t m, int64_t k, int64_t lda, const double2* X,
            int64_t R, double2* Y, int64_t ldy);
int df_combine(bem_ctx* ctx, const float4* B, const int* eB, int64_t K, int64_t n, const double2* W, int64_t R,
               double2* U);
}  // namespace gbem
