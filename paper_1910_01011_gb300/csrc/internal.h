// internal.h -- data layout shared by the library's translation units.
//
// Triangles are stored tile-ordered: each domain's triangles are sorted
// along a Morton curve of their centroids and cut into tiles of TT
// triangles (the last tile of a domain is padded).  A tile carries its
// centre in FP64; every point and plane offset of the tile is stored
// relative to that centre, so FP32 differences between points of two tiles
// keep their accuracy (the far-field phase is reconstructed from an FP64
// tile-pair distance plus an FP32 local offset).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/bem.h"

namespace gbem {

constexpr int TT = 32;          // triangles per tile
constexpr int QP = 6;           // regular-rule points per triangle
constexpr int TP = TT * QP;     // points per tile = threads of a far-field CTA
constexpr int NCOMP = 14;       // potentials per target point and wavenumber slot
constexpr int CHUNK_MAX = 256;  // source tiles per far-field CTA (shared-memory table bound)

// ------------------------------------------------------------------ host geometry

struct Quadrature {
    double l1[QP], l2[QP], w[QP];  // regular rule (weights sum to 1)
    double lam[QP][3];             // P1 values at the rule points
    int ng = 6;                    // Gauss points per singular direction
    // point tables per relation (0 near pair: collapsed Gauss-Legendre on each
    // triangle; 1 vertex, 2 edge, 3 identical: Sauter-Schwab):
    // rows (s1, s2, t1, t2, weight * jacobian)
    std::vector<double> ss[4];
};

struct HostDomain {
    std::vector<double> verts;   // nv*3
    std::vector<int32_t> tris;   // nt*3
    int64_t nv = 0, nt = 0;
    double kre = 0, kim = 0, rho = 1;
};

struct Geometry {
    int n_dom = 0;
    int n_tiles = 0;
    int64_t n_slots = 0, n_pts = 0, n_vert = 0, n_dof = 0, n_tri = 0;
    std::vector<int> dom_tile_begin, dom_tile_end;
    std::vector<int64_t> dom_vert_off, dom_dof_off, dom_nv;
    // per tile
    std::vector<double> tile_c;     // 4 per tile (x, y, z, radius)
    std::vector<int> tile_dom, tile_ntri;
    // per triangle slot (tile order, padded)
    std::vector<int> slot_v;        // 4 per slot: global vertex ids (pad: -1), domain
    std::vector<double> slot_P;     // 9 per slot: absolute vertex coordinates
    std::vector<double> slot_n;     // 3 per slot: unit normal
    std::vector<double> slot_area;  // 1 per slot
    std::vector<double> slot_curl;  // 9 per slot: surface curls of the 3 P1 functions
    std::vector<double> slot_h;     // n . (P0 - tile centre)
    // per point
    std::vector<double> pt_delta;   // 3 per point, relative to the tile centre
    std::vector<double> pt_w;       // rule weight * area (0 for padding)
    // vertex -> corner CSR (corner = slot*3 + local vertex)
    std::vector<int64_t> vc_ptr;
    std::vector<int32_t> vc_idx;
    std::vector<int64_t> v_dof1, v_dof2;  // system index of psi (row1) and phi (row2) of a vertex
    // touching pairs, CSR over target slots
    std::vector<int64_t> np_ptr;
    std::vector<int32_t> np_src;
    std::vector<int32_t> np_code;   // rel | pa0<<4 | pa1<<6 | pa2<<8 | pb0<<10 | pb1<<12 | pb2<<14
    double max_diameter = 0;        // largest domain bounding-box diagonal
};

// Derive the regular 6-point rule (moment equations), Gauss-Legendre nodes
// and the Sauter-Schwab tables.  Returns false on a Newton failure.
bool build_quadrature(Quadrature& q, int n_gauss);
bool gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);

// Validate the meshes and build the tiled geometry.  Returns an empty string
// on success, else the error message.
std::string build_geometry(const std::vector<HostDomain>& doms, const Quadrature& q, Geometry& g);

// ------------------------------------------------------------------ device views

// Pair-interleaved storage of the QP points of one triangle, the layout in
// which the FP32 far field reads its sources (two points per packed FP32
// instruction): pair j (points 2j and 2j+1) is the float4
// (x_a, x_b, y_a, y_b) at 2j followed by (z_a, z_b, w_a, w_b) at 2j + 1.
static_assert(QP % 2 == 0, "points pair up within a triangle");
__host__ __device__ inline void pair_interleave(const float4 (&pt)[QP], float4* out) {
    for (int j = 0; j < QP / 2; j++) {
        const float4 a = pt[2 * j], b = pt[2 * j + 1];
        out[2 * j] = make_float4(a.x, b.x, a.y, b.y);
        out[2 * j + 1] = make_float4(a.z, b.z, a.w, b.w);
    }
}
// Point q of a triangle stored pair-interleaved at tri.
__host__ __device__ inline float4 pair_point(const float4* tri, int q) {
    const float4 u = tri[q & ~1], v = tri[(q & ~1) + 1];
    return (q & 1) ? make_float4(u.y, u.w, v.y, v.w) : make_float4(u.x, u.z, v.x, v.z);
}

struct FarArgs32 {
    const float4* pg;       // [n_pts]   (dx, dy, dz, w)          target points
    const float4* pgp;      // [n_pts]   the same, pair-interleaved  source points
    const float4* tg;       // [n_slots] (nx, ny, nz, h)
    const double4* tc;      // [n_tiles] centre
    const int* tdom;        // [n_tiles]
    const int* tntri;       // [n_tiles]
    const float4* pd;       // [n_pts]   (sigN re, im, sigD re, im) * w, pair-interleaved
    const float4* tcurl;    // [2*n_slots] (Cre, 0), (Cim, 0)
    const int2* dom_tiles;  // [n_dom] own-domain tile range (slot 1 sources)
    const double2* kdom;    // [n_dom] slot-1 wavenumber
    double2 k0;             // slot-0 wavenumber
    int src_begin, src_end; // slot-0 source tiles
    int tgt_begin;          // first target tile (grid.x offset)
    int chunk_tiles;        // source tiles per grid.y index
    int slot1;              // 1: interior wavenumber on own-domain sources
    int64_t n_pts;          // points per (chunk, slot, component) row of partial
    int64_t p_off;          // point number stored at column 0 of partial (0 unless a caller batches targets)
    float* partial;         // [grid.y][2][NCOMP][n_pts], column p - p_off for point p
    int* err;               // device error flag (bounded waits)
    const int2* work;       // null: grid (target tiles, chunks); else [n_work] (target tile offset, chunk)
                            // in launch order, heaviest first, on a 1-D grid
};

// Several right-hand sides in one far-field launch: work item
// (target tile offset, source chunk, wavenumber slot, group of MRG right-hand
// sides).  Right-hand side r has its own densities (pd + r * n_pts,
// tcurl + r * 2 * n_slots) and its own partial buffer (partial + r * rstride,
// laid out as for one right-hand side).
constexpr int MRG = 4;
struct FarArgs32M {
    const float4* pg;       // target points
    const float4* pgp;      // source points, pair-interleaved
    const float4* tg;
    const double4* tc;
    const int* tdom;
    const int* tntri;
    const float4* pd;       // [R][n_pts] densities, pair-interleaved
    const float4* tcurl;    // [R][2 * n_slots]
    const int2* dom_tiles;
    const double2* kdom;
    double2 k0;
    int src_begin, src_end, tgt_begin, chunk_tiles;
    int R;
    int64_t n_pts, n_slots;
    int64_t rstride;        // floats between the partial buffers of consecutive right-hand sides
    float* partial;         // [R][n_chunks][2][NCOMP][n_pts]
    int* err;
    const int4* work;       // [n_work] (target tile offset, chunk, slot, group), heaviest first
};

struct FarArgs64 {
    const double4* pg;      // (dx, dy, dz, w)
    const double4* tg;      // (nx, ny, nz, h)
    const double4* tc;
    const int* tdom;
    const int* tntri;
    const double4* pd;      // (sigN re, im, sigD re, im) * w
    const double4* tcurl;   // [2*n_slots] (Cre, 0), (Cim, 0)
    const int2* dom_tiles;
    const double2* kdom;
    double2 k0;
    int src_begin, src_end, tgt_begin, chunk_tiles, slot1;
    int64_t n_pts;
    double* partial;
};

// Several vectors in one FP64 far-field launch (far64m_kernel): CTA (x, y, z)
// = (target tile, source chunk, slot x group); slot 0 sums every source tile
// of the chunk at k0, slot 1 the target domain's own tiles at k_j (PMCHWT),
// a group is RG64 consecutive vectors.
constexpr int RG64 = 4;
struct FarArgs64M {
    const double4* pg;      // (dx, dy, dz, w)
    const double4* tg;      // (nx, ny, nz, h)
    const double4* tc;
    const int* tdom;
    const int* tntri;
    const double4* pd;      // [R][n_pts] (sigN re, im, sigD re, im) * w
    const double4* tcurl;   // [R][2 n_slots]
    const int2* dom_tiles;
    const double2* kdom;
    double2 k0;
    int src_begin, src_end, tgt_begin, chunk_tiles, slot1, groups, R;
    int64_t n_pts, n_slots, rstride;  // rstride: doubles between consecutive vectors' partials
    double* partial;        // [R][n_chunks][2][NCOMP][n_pts]
};
cudaError_t launch_far64_multi(const FarArgs64M& a, int n_tgt_tiles, int n_chunks, cudaStream_t s);

// Split constants of the double-float sin, cos and exp (df_math.cuh): pi/64
// in four FP32 parts, ln2/64 in three, 64/pi, 64/ln2 and -1/6 as (h, l).
struct DfConsts {
    float pi64[4], ln64[3], inv_pi64, inv_ln64, sixth[2];
};

// The far field to FP64 accuracy in double-float FP32 arithmetic (k_fardf.cu):
// the same work decomposition as FarArgs64M, every real as an (h, l) pair of
// floats (geometry split once, densities split per call with a power-of-two
// scale per vector).
struct FarArgsDF {
    const float4 *pgh, *pgl;   // [n_pts] point offset from its tile centre, weight
    const float4 *tgh, *tgl;   // [n_slots] normal, h
    const float4 *tch, *tcl;   // [n_tiles] tile centres
    const int* tdom;
    const int* tntri;
    const int2* dom_tiles;
    const float4* kdf;         // [n_dom] (Re k hi, lo, Im k hi, lo) of each domain
    float4 k0df;               // slot-0 wavenumber
    const float4 *pdh, *pdl;   // [R][n_pts] scaled densities
    const float4 *cuh, *cul;   // [R][2 n_slots] scaled curls
    const int* vexp;           // [R] each vector's scale is 2^-vexp
    const float4* sctab;       // [128] (sin hi, lo, cos hi, lo) of j pi / 64
    const float2* extab;       // [64] 2^(-j/64) hi, lo
    DfConsts c;                // split constants of the double-float sin, cos and exp
    int src_begin, src_end, tgt_begin, chunk_tiles, slot1, groups, R;
    int64_t n_pts, n_slots, rstride;
    double* partial;           // [R][n_chunks][2][NCOMP][n_pts]
};

struct GatherArgs {
    const int4* slot_v;         // [n_slots] vertex ids (-1 pad), .w = domain
    const int64_t* v_dof1;      // per global vertex
    const int64_t* v_dof2;
    const double* pt_w;         // [n_pts]
    const double* slot_curl;    // [n_slots*9]
    const double2* x;           // system-order input
    int64_t s_begin, s_end;     // slots to gather
    double lam[QP][3];          // P1 values at the rule points
    float4* pd32; float4* tcurl32;     // fp32 outputs (may be null); pd32 pair-interleaved
    double4* pd64; double4* tcurl64;   // fp64 outputs (may be null)
};

struct SlotCoef {               // per (domain, slot): row coefficients
    double cV, cK, cKp, cW;
    double k2re, k2im;          // k^2 of the slot
};

struct ProjectArgs {
    const int4* slot_v;
    const double* pt_w;
    const double* slot_curl;
    const int* tntri;
    const int* tdom;
    const SlotCoef* coef;       // [n_dom*2]
    int tgt_begin, tgt_end;     // target tiles
    int n_chunks;
    int64_t n_pts;
    int64_t p_off;              // point number at column 0 of the partials (as FarArgs32::p_off)
    const float* partial32;     // one of the two is non-null
    const double* partial64;
    // touching-pair correction (may be empty)
    const int64_t* np_ptr;      // [n_slots+1]
    const int32_t* np_src;
    const double2* nb64;        // [pair][4][9] combined sub-blocks, FP64
    const float2* nb32;         // FP32 copy (used by the FP32 path)
    const int64_t* v_dof1;
    const int64_t* v_dof2;
    const double2* x;           // input vector (system order)
    double2* tri_out;           // [n_slots*3][2] per-corner rows
    double lam[QP][3];
};

struct ReduceArgs {
    const int64_t* vc_ptr;
    const int32_t* vc_idx;
    const int64_t* v_dof1;
    const int64_t* v_dof2;
    const double2* tri_out;
    int64_t v_begin, v_end;     // global vertices to produce
    double2* y;
};

struct NearArgs {
    int64_t n_pairs;
    const int32_t* pair_tgt;    // target slot of each pair
    const int32_t* pair_src;
    const int32_t* pair_code;
    const double* slot_P;       // [n_slots*9]
    const double* slot_n;       // [n_slots*3]
    const double* slot_area;
    const double* slot_curl;
    const double* ss_tab[4];    // device Sauter-Schwab tables (5 doubles per point)
    int ss_n[4];
    double rule[3 * QP];        // regular rule (l1, l2, w)
    double2 k[2];               // slot wavenumbers: slot 0, slot 1 (per target domain: kdom)
    const double2* kdom;
    const int* slot_dom;        // via slot_v.w
    int n_slot_k;               // 1 or 2
    double2* raw;               // [pair][slot][27]: V, K, K' (SS minus regular)
    // double-float point evaluations (use_df): tables as (hi, lo) floats,
    // sin / cos / exp tables and constants, wavenumbers, regular rule, 1 / (4 pi)
    int use_df;
    const float* ss_tabf[4];
    const float4* sctab;
    const float2* extab;
    DfConsts c;
    const float4* kdf;
    float4 k0df;
    float rule_h[3 * QP], rule_l[3 * QP];
    float i4h, i4l;
};

struct NearCombineArgs {
    int64_t n_pairs;
    const int32_t* pair_tgt;
    const int32_t* pair_src;
    const double* slot_n;
    const double* slot_curl;
    const int4* slot_v;
    const SlotCoef* coef;       // [n_dom*2]
    int n_slot_k;
    const double2* raw;
    double2* nb64;
    float2* nb32;
};

// launchers (k_apply.cu, k_near.cu)
cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s);
cudaError_t launch_far32(const FarArgs32& a, int n_tgt_tiles, int n_chunks, cudaStream_t s);
cudaError_t launch_far32_group(const FarArgs32* group, const int4* gwork, int64_t n_work, cudaStream_t s);
cudaError_t launch_far32_multi(const FarArgs32M& a, int64_t n_work, cudaStream_t s);
cudaError_t launch_far64(const FarArgs64& a, int n_tgt_tiles, int n_chunks, cudaStream_t s);
cudaError_t launch_project(const ProjectArgs& a, cudaStream_t s);
cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t s);
cudaError_t launch_near_build(const NearArgs& a, cudaStream_t s);
cudaError_t launch_near_combine(const NearCombineArgs& a, cudaStream_t s);
size_t far32_smem_bytes();

}  // namespace gbem
