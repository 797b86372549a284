// k_gemm.cu -- complex64 matrix x block of vectors on the 5th-generation
// tensor cores (tcgen05), split BF16 with FP32 accumulation.
//
// Y = A X with A (m x k) and X (k x n) complex.  Each real plane P of A and
// of X is split into three BF16 numbers, P ~ P0 + P1 + P2 with
// P0 = bf16(P), P1 = bf16(P - P0), P2 = bf16(P - P0 - P1), and the product
// keeps the six terms Pi Qj with i + j <= 2 (everything down to ~2^-24 of
// the product, FP32 level).  A two-term split (three products, ~2^-17 per
// term) is not enough for the oscillatory high-frequency operators: its
// per-term error is amplified by the cancellation in A x (measured 1.2e-4
// on the 0.5 MHz rib scene against 2e-6 for the FP32 matrix-free path).
//
// The complex product is two real GEMMs sharing the B operand
// B = [X_re | X_im] (k x 2n):  C1 = A_re B,  C2 = A_im B, then
//   Y_re = C1[:, :n] - C2[:, n:],   Y_im = C1[:, n:] + C2[:, :n].
// A CTA owns a 128-row tile of A and a 128-column tile of B (64 right-hand
// sides, real and imaginary parts), so C1 and C2 are two 128 x 128 FP32
// accumulators in tensor memory (256 TMEM columns, double-buffered over 512).
// Operands stream in by TMA (64-byte swizzle, K-major, 32 of K per stage)
// through a three-stage ring (GSTAGES); one thread issues the MMAs and
// commits each stage back to the producer.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>
#include <string>

#include "ctx.h"
#include "internal.h"

namespace gbem {

constexpr int GM = 128;                       // rows of A per CTA
constexpr int GN = 128;                       // columns of B per CTA (64 rhs x re/im)
constexpr int GK = 32;                        // k per stage (64 bytes of bf16, 64-byte swizzle)
constexpr int NSPLIT = 3;                     // BF16 terms per real number
constexpr int GSTAGES = 3;
constexpr int TILE_BYTES = GM * GK * 2;       // 8 KB per operand tile
constexpr int A_TILES = 2 * NSPLIT;           // A re (3 terms), A im (3 terms)
constexpr int G_STAGE_BYTES = (A_TILES + NSPLIT) * TILE_BYTES;
constexpr int GEMM_THREADS = 192;             // warp 0 TMA, warp 1 MMA, warps 2-5 accumulate / epilogue
constexpr uint32_t TMEM_COLS = 512;           // two accumulator buffers of 256 columns (C1 | C2)
constexpr int KCH_STAGES = 8;                 // stages per accumulation chunk (K = 256)

struct GemmSmem {
    alignas(1024) uint8_t stage[GSTAGES][G_STAGE_BYTES];
    uint64_t full[GSTAGES];
    uint64_t empty[GSTAGES];
    uint64_t accf[2];   // chunk accumulated in TMEM buffer b (MMA commit)
    uint64_t acce[2];   // TMEM buffer b drained (4 epilogue warps)
    uint32_t tmem_base;
};

__device__ __forceinline__ uint32_t s_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void g_mbar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void g_mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ uint32_t g_mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(s_u32(b)), "r"(parity)
        : "memory");
    return ok;
}
// Bounded wait (about a second); on timeout raise the error flag and return false.
__device__ __forceinline__ bool g_mbar_wait(uint64_t* b, uint32_t parity, int* err) {
    if (g_mbar_try(b, parity)) return true;
    if (*(volatile int*)err) return false;  // an earlier wait already gave up: do not wait again
    const long long t0 = clock64();
    while (!g_mbar_try(b, parity)) {
        if (clock64() - t0 > (1ll << 31)) {
            atomicExch(err, 2);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(s_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(s_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, rows of
// 64 bytes, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);           // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(512 >> 4) << 32;                 // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)4 << 61;                          // 64-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: BF16 A and B, FP32 D, both K-major,
// M = 128, N = 128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GN >> 3) << 17) | ((uint32_t)(GM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// The tensor cores accumulate FP32 with truncation, so a long K sum drifts
// by ~K x 2^-24 relative.  The MMAs therefore accumulate only KCH_STAGES*GK
// of K in tensor memory (two buffers, double-buffered); four epilogue warps
// drain each chunk into round-to-nearest FP32 registers.
// grid: (n_col_tiles, m_tiles); the column tile runs fastest so that the
// CTAs sharing an A row tile run together and share it through L2.
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    gemm_bf16x3_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       int64_t mpad, int64_t nbpad, int kblocks, int m, int n_rhs, float2* Y, int* err) {
    extern __shared__ uint8_t smem_raw[];
    GemmSmem& sm = *reinterpret_cast<GemmSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ct = blockIdx.x, mt = blockIdx.y;
    const int m0 = mt * GM;
    const int b0 = ct * GN;  // B rows (rhs re block then rhs im block)
    const int nchunks = (kblocks + KCH_STAGES - 1) / KCH_STAGES;

    if (threadIdx.x == 0) {
        for (int s = 0; s < GSTAGES; s++) {
            g_mbar_init(&sm.full[s], 1);
            g_mbar_init(&sm.empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            g_mbar_init(&sm.accf[b], 1);
            g_mbar_init(&sm.acce[b], 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&sm.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = sm.tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // producer
            for (int kb = 0; kb < kblocks; kb++) {
                const int s = kb % GSTAGES, u = kb / GSTAGES;
                if (kb >= GSTAGES && !g_mbar_wait(&sm.empty[s], (uint32_t)((u - 1) & 1), err)) break;
                uint8_t* st = sm.stage[s];
                g_mbar_expect_tx(&sm.full[s], G_STAGE_BYTES);
                const int kx = kb * GK;
                for (int pl = 0; pl < A_TILES; pl++)
                    tma_2d(st + pl * TILE_BYTES, &tmA, kx, (int)(pl * mpad + m0), &sm.full[s]);
                for (int pl = 0; pl < NSPLIT; pl++)
                    tma_2d(st + (A_TILES + pl) * TILE_BYTES, &tmB, kx, (int)(pl * nbpad + b0), &sm.full[s]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: per chunk, buffer b: C1 (cols 256b..256b+127) = A_re B,
            // C2 (256b+128..256b+255) = A_im B, each as the six products A_i B_j, i + j <= 2
            bool ok = true;
            for (int kb = 0; kb < kblocks && ok; kb++) {
                const int c = kb / KCH_STAGES, first = (kb % KCH_STAGES) == 0;
                const int buf = c & 1;
                const uint32_t acc_base = tmem + (uint32_t)(buf * 256);
                if (first && c >= 2) {
                    ok = g_mbar_wait(&sm.acce[buf], (uint32_t)(((c >> 1) - 1) & 1), err);
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                }
                const int s = kb % GSTAGES, u = kb / GSTAGES;
                ok = ok && g_mbar_wait(&sm.full[s], (uint32_t)(u & 1), err);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = s_u32(sm.stage[s]);
#pragma unroll
                for (int kk = 0; kk < GK / 16; kk++) {
                    const uint32_t off = kk * 32;
                    uint64_t ar[NSPLIT], ai[NSPLIT], bd[NSPLIT];
#pragma unroll
                    for (int t = 0; t < NSPLIT; t++) {
                        ar[t] = smem_desc(base + t * TILE_BYTES + off);
                        ai[t] = smem_desc(base + (NSPLIT + t) * TILE_BYTES + off);
                        bd[t] = smem_desc(base + (A_TILES + t) * TILE_BYTES + off);
                    }
                    const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
                    mma_bf16(acc_base, ar[0], bd[0], acc);
                    mma_bf16(acc_base, ar[0], bd[1], 1u);
                    mma_bf16(acc_base, ar[1], bd[0], 1u);
                    mma_bf16(acc_base, ar[0], bd[2], 1u);
                    mma_bf16(acc_base, ar[1], bd[1], 1u);
                    mma_bf16(acc_base, ar[2], bd[0], 1u);
                    mma_bf16(acc_base + 128, ai[0], bd[0], acc);
                    mma_bf16(acc_base + 128, ai[0], bd[1], 1u);
                    mma_bf16(acc_base + 128, ai[1], bd[0], 1u);
                    mma_bf16(acc_base + 128, ai[0], bd[2], 1u);
                    mma_bf16(acc_base + 128, ai[1], bd[1], 1u);
                    mma_bf16(acc_base + 128, ai[2], bd[0], 1u);
                }
                mma_commit(&sm.empty[s]);
                if ((kb % KCH_STAGES) == KCH_STAGES - 1 || kb == kblocks - 1) mma_commit(&sm.accf[buf]);
            }
            // a chunk cut short by a timeout still signals its buffer
            if (!ok) {
                mma_commit(&sm.accf[0]);
                mma_commit(&sm.accf[1]);
            }
        }
    } else {
        // accumulate each chunk (round-to-nearest FP32) and write Y
        const int q = warp & 3;  // TMEM lane quarter this warp may access
        const int row = m0 + q * 32 + lane;
        float yr[64], yi[64];
#pragma unroll
        for (int j = 0; j < 64; j++) yr[j] = yi[j] = 0.f;
        for (int c = 0; c < nchunks; c++) {
            const int buf = c & 1;
            g_mbar_wait(&sm.accf[buf], (uint32_t)((c >> 1) & 1), err);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t lb = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 256);
#pragma unroll
            for (int jc = 0; jc < 64; jc += 16) {
                float ta[16], tb[16];
                tmem_ld16(lb + jc, ta);         // A_re X_re
                tmem_ld16(lb + 192 + jc, tb);   // A_im X_im
#pragma unroll
                for (int j = 0; j < 16; j++) yr[jc + j] += ta[j] - tb[j];
                tmem_ld16(lb + 64 + jc, ta);    // A_re X_im
                tmem_ld16(lb + 128 + jc, tb);   // A_im X_re
#pragma unroll
                for (int j = 0; j < 16; j++) yi[jc + j] += ta[j] + tb[j];
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(&sm.acce[buf])) : "memory");
        }
        if (row < m) {
#pragma unroll
            for (int j = 0; j < 64; j++) {
                const int rhs = ct * 64 + j;
                if (rhs < n_rhs) Y[(int64_t)rhs * m + row] = make_float2(yr[j], yi[j]);
            }
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 2) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// x -> three BF16 terms, x ~ t0 + t1 + t2
__device__ __forceinline__ void split3(float x, __nv_bfloat16& t0, __nv_bfloat16& t1, __nv_bfloat16& t2) {
    t0 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(t0);
    t1 = __float2bfloat16_rn(r1);
    t2 = __float2bfloat16_rn(r1 - __bfloat162float(t1));
}

// A (m x k, complex64 row-major) -> bf16 planes [re0, re1, re2, im0, im1, im2][mpad][kpad], zero padded
__global__ void split_a_kernel(const float2* A, int64_t m, int64_t k, int64_t mpad, int64_t kpad, __nv_bfloat16* P) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= mpad * kpad) return;
    const int64_t r = idx / kpad, c = idx % kpad;
    float2 v = make_float2(0.f, 0.f);
    if (r < m && c < k) v = A[r * k + c];
    const int64_t plane = mpad * kpad;
    split3(v.x, P[0 * plane + idx], P[1 * plane + idx], P[2 * plane + idx]);
    split3(v.y, P[3 * plane + idx], P[4 * plane + idx], P[5 * plane + idx]);
}

// X (n_rhs x k, complex64, rhs-major) -> bf16 planes [t0, t1, t2][nbpad][kpad];
// B row of rhs j, part p (0 re, 1 im) = (j / 64) * 128 + p * 64 + j % 64.
__global__ void split_x_kernel(const float2* X, int64_t n_rhs, int64_t k, int64_t nbpad, int64_t kpad,
                               __nv_bfloat16* P) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nbpad * kpad) return;
    const int64_t brow = idx / kpad, c = idx % kpad;
    const int64_t blk = brow / 128, within = brow % 128, part = within / 64, j = blk * 64 + within % 64;
    float x = 0.f;
    if (j < n_rhs && c < k) {
        const float2 v = X[j * k + c];
        x = part ? v.y : v.x;
    }
    split3(x, P[idx], P[nbpad * kpad + idx], P[2 * nbpad * kpad + idx]);
}

// Resolved once (thread-safe static initialisation; contexts on several
// threads share it).
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000)p;
        return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }();
    return fn;
}

static bool make_map(CUtensorMap* map, void* base, int64_t rows, int64_t kpad) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
    cuuint32_t box[2] = {GK, GM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Planes of A are kept by the caller (they are the assembled operator); X
// is split per call.  Y (n_rhs x m complex64) = A X.
int gemm_bf16x3(bem_ctx* ctx, const __nv_bfloat16* Aplanes, int64_t m, int64_t k, int64_t mpad, int64_t kpad,
                const float2* X, int64_t n_rhs, float2* Y, __nv_bfloat16* xplanes, int64_t nbpad) {
    static_assert(sizeof(GemmSmem) <= 227 * 1024 - 1024, "gemm smem");
    CUtensorMap ta, tb;
    if (!make_map(&ta, (void*)Aplanes, A_TILES * mpad, kpad) || !make_map(&tb, (void*)xplanes, NSPLIT * nbpad, kpad))
        return ctx->fail(BEM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    const int64_t nx = nbpad * kpad;
    split_x_kernel<<<(unsigned)((nx + 255) / 256), 256, 0, ctx->stream>>>(X, n_rhs, k, nbpad, kpad, xplanes);
    const size_t smem = sizeof(GemmSmem) + 1024;
    static const cudaError_t attr_e =
        cudaFuncSetAttribute(gemm_bf16x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr_e != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string("gemm attribute: ") + cudaGetErrorString(attr_e));
    const dim3 grid((unsigned)(nbpad / GN), (unsigned)(mpad / GM));
    gemm_bf16x3_kernel<<<grid, GEMM_THREADS, smem, ctx->stream>>>(ta, tb, mpad, nbpad, (int)(kpad / GK), (int)m,
                                                                  (int)n_rhs, Y, ctx->dev.err);
    ctx->launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string("gemm launch: ") + cudaGetErrorString(e));
    return BEM_OK;
}

int gemm_a_planes() { return A_TILES; }
int gemm_b_planes() { return NSPLIT; }
int gemm_k_align() { return GK; }

int split_a(bem_ctx* ctx, const float2* A, int64_t m, int64_t k, int64_t mpad, int64_t kpad, __nv_bfloat16* P) {
    const int64_t n = mpad * kpad;
    split_a_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(A, m, k, mpad, kpad, P);
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, std::string("split_a: ") + cudaGetErrorString(e));
    return BEM_OK;
}

}  // namespace gbem

using namespace gbem;

// Test/utility entry: Y = A X for device complex64 arrays (see bem.h).
extern "C" int bem_zgemm_bf16x3(bem_ctx* ctx, int64_t m, int64_t k, int64_t n_rhs, const void* A, const void* X,
                                void* Y) {
    if (!ctx) return BEM_ERR_INVALID_ARG;
    if (m < 1 || k < 1 || n_rhs < 1 || !A || !X || !Y) return ctx->fail(BEM_ERR_INVALID_ARG, "bad gemm arguments");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ctx->fail(BEM_ERR_CUDA, "cudaSetDevice");
    if (!ctx->dev.err) {
        int rc;
        ctx->dev.err = (int*)ctx->dalloc(sizeof(int), &rc);
        if (rc) return rc;
        cudaMemsetAsync(ctx->dev.err, 0, sizeof(int), ctx->stream);
    }
    const int64_t mpad = (m + GM - 1) / GM * GM, kpad = (k + GK - 1) / GK * GK;
    const int64_t nbpad = (n_rhs + 63) / 64 * 128;
    int rc;
    __nv_bfloat16* ap = (__nv_bfloat16*)ctx->dalloc((size_t)A_TILES * mpad * kpad * 2, &rc);
    if (rc) return rc;
    __nv_bfloat16* xp = (__nv_bfloat16*)ctx->dalloc((size_t)NSPLIT * nbpad * kpad * 2, &rc);
    if (rc) { ctx->dfree(ap); return rc; }
    rc = split_a(ctx, (const float2*)A, m, k, mpad, kpad, ap);
    if (!rc) rc = gemm_bf16x3(ctx, ap, m, k, mpad, kpad, (const float2*)X, n_rhs, (float2*)Y, xp, nbpad);
    cudaStreamSynchronize(ctx->stream);
    ctx->dfree(ap);
    ctx->dfree(xp);
    if (!rc) rc = ctx->check_device_error();
    return rc;
}
