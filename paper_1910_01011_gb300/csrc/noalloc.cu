// noalloc.cu -- an allocation-free variant of the FP32 operator application.
//
// bem_apply may allocate device memory on first use (the far-field kernel's
// per-chunk partial potentials grow with the problem).  Some callers cannot
// let the library call cudaMalloc at that point: a process whose device
// memory is fully reserved by another allocator (for example a framework's
// caching pool), or a latency-critical loop that must never enter the CUDA
// allocator.  bem_apply_noalloc serves them: it keeps the far-field scratch
// in the fixed array below instead of allocating it, and processes the
// target tiles in batches sized to fit that array.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "ctx.h"
#include "internal.h"

using namespace gbem;

// Scratch of the allocation-free apply: 64 MiB of FP32 partial potentials.
// It is part of the library's device image, so every GPU that loads the
// library holds it until the process exits.  All calls share it.
constexpr size_t NOALLOC_SCRATCH_FLOATS = (size_t)16 << 20;
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_SCRATCH_FLOATS];

// Device address of g_noalloc_scratch per device, looked up once per device
// (with that device current).  In host code the symbol itself is only a
// host-side stand-in and must never be handed to a kernel.
static float* g_scratch_addr[128] = {};
static std::mutex g_scratch_mu;

static int scratch_for_device(bem_ctx* ctx, float** out) {
    if (ctx->device < 0 || ctx->device >= 128) return ctx->fail(BEM_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[ctx->device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return ctx->fail(BEM_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_addr[ctx->device] = (float*)p;
    }
    *out = g_scratch_addr[ctx->device];
    return BEM_OK;
}

#define CK(expr)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" int bem_apply_noalloc(bem_ctx* ctx, const bem_z* x, bem_z* y) {
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (!x || !y) return ctx->fail(BEM_ERR_INVALID_ARG, "null vector");
    if (!ctx->ready || !ctx->near_ready)
        return ctx->fail(BEM_ERR_STATE,
                         "bem_apply_noalloc needs a prepared context: call bem_apply once (it allocates) first");
    CK(cudaSetDevice(ctx->device));
    float* scratch = nullptr;
    int rc = scratch_for_device(ctx, &scratch);
    if (rc) return rc;
    const Geometry& g = ctx->geo;
    const int n_tiles = g.n_tiles;
    int n_chunks, chunk_tiles;
    ctx->chunking(n_tiles, n_tiles, &n_chunks, &chunk_tiles);
    const size_t per_tile = (size_t)n_chunks * 2 * NCOMP * TP;  // floats of scratch per target tile
    if (per_tile > NOALLOC_SCRATCH_FLOATS)
        return ctx->fail(BEM_ERR_OUT_OF_BUDGET, "problem too large for the 64 MiB allocation-free scratch (" +
                                                    std::to_string(n_chunks) + " source chunks per target tile)");
    const int batch = (int)std::min<size_t>((size_t)n_tiles, NOALLOC_SCRATCH_FLOATS / per_tile);
    const double2* xd = (const double2*)x;
    double2* yd = (double2*)y;
    // trial densities of every source tile (context-owned buffers)
    GatherArgs ga{};
    ga.slot_v = ctx->dev.slot_v;
    ga.v_dof1 = ctx->dev.v_dof1;
    ga.v_dof2 = ctx->dev.v_dof2;
    ga.pt_w = ctx->dev.pt_w;
    ga.slot_curl = ctx->dev.slot_curl;
    ga.x = xd;
    ga.s_begin = 0;
    ga.s_end = g.n_slots;
    for (int q = 0; q < QP; q++)
        for (int k = 0; k < 3; k++) ga.lam[q][k] = ctx->quad.lam[q][k];
    ga.pd32 = ctx->dev.pd32;
    ga.tcurl32 = ctx->dev.tcurl32;
    CK(launch_gather(ga, ctx->stream));
    for (int tb = 0; tb < n_tiles; tb += batch) {
        const int te = std::min(n_tiles, tb + batch);
        const int64_t stride = (int64_t)(te - tb) * TP;
        // The scratch holds the batch's points only: point p of the batch is
        // column p - p_off of each (chunk, slot, component) row of length stride.
        const int64_t p_off = (int64_t)tb * TP;
        FarArgs32 fa{};
        fa.pg = ctx->dev.pg32; fa.pgp = ctx->dev.pgp32; fa.tg = ctx->dev.tg32; fa.tc = ctx->dev.tc; fa.tdom = ctx->dev.tdom;
        fa.tntri = ctx->dev.tntri; fa.pd = ctx->dev.pd32; fa.tcurl = ctx->dev.tcurl32;
        fa.dom_tiles = ctx->dev.dom_tiles; fa.kdom = ctx->dev.kdom;
        fa.k0 = make_double2(ctx->k0re, ctx->k0im);
        fa.src_begin = 0; fa.src_end = n_tiles; fa.tgt_begin = tb; fa.chunk_tiles = chunk_tiles; fa.slot1 = 1;
        fa.n_pts = stride; fa.p_off = p_off; fa.partial = scratch; fa.err = ctx->dev.err;
        CK(launch_far32(fa, te - tb, n_chunks, ctx->stream));
        ProjectArgs pa{};
        pa.slot_v = ctx->dev.slot_v; pa.pt_w = ctx->dev.pt_w; pa.slot_curl = ctx->dev.slot_curl;
        pa.tntri = ctx->dev.tntri; pa.tdom = ctx->dev.tdom; pa.coef = ctx->dev.coef;
        pa.tgt_begin = tb; pa.tgt_end = te; pa.n_chunks = n_chunks; pa.n_pts = stride; pa.p_off = p_off; pa.partial32 = scratch;
        if (ctx->pmchwt_near.n_pairs > 0) {
            pa.np_ptr = ctx->dev.np_ptr; pa.np_src = ctx->dev.np_src; pa.nb32 = ctx->pmchwt_near.nb32;
        }
        pa.v_dof1 = ctx->dev.v_dof1; pa.v_dof2 = ctx->dev.v_dof2; pa.x = xd; pa.tri_out = ctx->dev.tri_out;
        for (int q = 0; q < QP; q++)
            for (int k = 0; k < 3; k++) pa.lam[q][k] = ctx->quad.lam[q][k];
        CK(launch_project(pa, ctx->stream));
    }
    ReduceArgs ra{};
    ra.vc_ptr = ctx->dev.vc_ptr; ra.vc_idx = ctx->dev.vc_idx; ra.v_dof1 = ctx->dev.v_dof1;
    ra.v_dof2 = ctx->dev.v_dof2; ra.tri_out = ctx->dev.tri_out; ra.y = yd; ra.v_begin = 0; ra.v_end = g.n_vert;
    CK(launch_reduce(ra, ctx->stream));
    return BEM_OK;
}
