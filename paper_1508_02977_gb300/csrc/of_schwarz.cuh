// Overlapping Schwarz preconditioner (Section 3.2, Eq. schwarz), fused with
// the residual update of the Krylov loop.  One subdomain is solved by one CTA
// at a time; the grid is persistent (a few CTAs per SM walk the subdomain
// list) and streams the next subdomain's data in by TMA while the current one
// is swept.
//
// Subdomain i owns a tile T_x x T_y of nodes; its extended tile adds `o`
// node layers on every side that is not on the image boundary (the overlap
// Sigma_ij of Section 3.2).  The local problem is the global operator
// restricted to the extended tile with homogeneous Dirichlet values outside
// it (the algebraic form of the Dirichlet transmission condition on
// Gamma_ij) and the natural Neumann condition on the image boundary.  It is
// solved approximately by `s` symmetric 3-colour block SOR sweeps from zero
// (colours (x+y) mod 3 make the 7-point stencil conflict free; a visit of
// colour c sets z_n <- z_n + omega (D_n^{-1}(b_n - sum_m A_nm z_m) - z_n) for
// all its nodes at once; omega = 1 is block Gauss-Seidel).  Each visit's
// error propagator I - omega P_c is self-adjoint in the A inner product with
// norm <= 1 for 0 < omega < 2, and the colour order 0,1,2,1,0,1,2,1,0,... is
// a palindrome, so the sweep operator is symmetric and the preconditioner
// positive definite for any such omega.  For CG the preconditioner must be symmetric, so
// the subdomain right-hand side is the residual on the owned nodes only and
// only the owned part of the local solution is kept:
//   z = sum_i R~_i^T  A_i^{-1}(approx)  R~_i r        (R~_i: owned nodes)
// which is symmetric positive definite (block diagonal over owned tiles of
// SPD blocks).  With sweeps = 0 and overlap 0 it is node-block Jacobi.
//
// Element data ("cells"): per node (x, y), the square (x, y) gives two
// records, t=0 and t=1, each (h, w) with h = g_K / sqrt(24) of that triangle
// and w the alpha-weight of one edge leaving the node (t=0: the edge to
// (x+1,y); t=1: the edge to (x,y+1)).  They depend on the frames and alpha
// only, so k_cells forms them once per solve (FP16 for the FP32 path: the
// preconditioner only has to be one fixed SPD operator, and the diagonal
// blocks are formed from the same rounded values, so the sweeps are exact
// block Gauss-Seidel on the rounded local operator).  Outside the image the
// records are zero (TMA fills out-of-range boxes with zeros), so missing
// triangles contribute nothing.
//
// Per subdomain:
//  1. TMA (cp.async.bulk.tensor) brings the two cell planes over the
//     extended tile plus a one-node ring and the owned tiles of r and q into
//     one of two stages (one mbarrier each, bounded waits); the next
//     subdomain's copies are issued as soon as this one's setup is done, so
//     they stream in during its sweeps.
//  2. Each thread owns, per colour, the nodes of a host-built table that
//     gives the 32 lanes of a warp 32 distinct shared-memory banks; it forms
//     their LDL^T-factored 3x3 diagonal blocks and right-hand sides in
//     registers (r <- r - a q fused here).  The first colour step from z = 0
//     is block Jacobi, z_n = D_n^{-1} r_n, done right here for colour 0.
//  3. Sweeps: one block update per owned node and colour step,
//     z_n = D_n^{-1} (r_n - sum_K h_K (h_K . (z_j + z_k)) + sum_e w_e z_e);
//     the first colour-1 step skips the colour-2 neighbours (still zero).
//  4. Coalesced write-out of z and r on the owned tile, FP64 partials of
//     r.r and r.z, deterministic last-CTA reduction per pair.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>

#include "of_common.cuh"

namespace ofk {

// tensor maps of a pair: element records, r, q, z, and the paired records of
// the FP16 sweeps (of_schwarz_h2.cuh)
enum { TM_C0 = 0, TM_C1 = 1, TM_R = 2, TM_Q = 3, TM_Z = 4, TM_P0 = 5, TM_P1 = 6, TM_PER_PAIR = 7 };

struct SchwarzParams {
    const PairDesc* pairs;
    const int4* tiles;        // per work item: (pair, tile x, tile y, global tile index)
    int ntiles;               // work items of this launch
    const CUtensorMap* tmaps; // [batch][TM_PER_PAIR], 64-byte aligned
    const uint32_t* ntab;     // [3][npt][blockDim] node of each (colour, slot, thread): i | j << 16, or ~0
    PairScalars* sc;
    double* partial;          // [ntiles][2]
    unsigned* counter;        // one arrival counter per launch (reset by the last CTA)
    int npairs;               // pairs of the batch (the last CTA updates each one's scalars)
    int* err;                 // device error word (bit 0: TMA wait timed out)
    void* r;                  // inner residual planes (written back on owned nodes)
    void* z;                  // preconditioned residual planes (owned nodes)
    double lam;
    double omega;             // relaxation factor of the sweeps (1: block Gauss-Seidel)
    int Tx, Ty, ov, sweeps;
    int first;                // no r update (start of a pass): z = M r only
    int apply_only;           // of_precondition: z = M r, no scalars
    int nstage;               // 2: the next item streams in during this one; 1: after it
    long long spin_limit;     // bounded mbarrier wait, in clock64 cycles
    int use_cond;             // launched in the inner-loop graph: set its while condition
    int defer;                // two-level: leave the scalars to the coarse correction's kernel
    int tx_extra;             // test hook (0 in use): bytes each staging barrier expects beyond its
                              // copies, so that its bounded wait runs out
    int pq_fixed;             // FP16 sweeps, one pair: a = r.z / p.q from PairScalars::pq_fix, formed here
    cudaGraphConditionalHandle cond;
};

// Cell grid of a subdomain: columns from cx0 = x0 - sch_cpad(o) (even, so
// that TMA boxes of 8-byte records start 16-byte aligned) to at least the
// ring column x0 + T_x + o; rows from y0 - o - 1 to y0 + T_y + o.
__host__ __device__ inline int sch_cpad(int ov) { return (ov + 2) & ~1; }
__host__ __device__ inline int sch_rw(int Tx, int ov) { return (sch_cpad(ov) + Tx + ov + 1 + 1) & ~1; }
__host__ __device__ inline int sch_rh(int Ty, int ov) { return Ty + 2 * ov + 2; }

// One cell record: float path 4 halves (8 bytes), FP64 path 4 doubles.
template <typename R> struct CellT;
template <> struct CellT<float> { using type = uint2; static constexpr int units = 1; };
template <> struct CellT<double> { using type = double4_32a; static constexpr int units = 4; };
template <typename R> __host__ __device__ constexpr int cell_bytes() { return (int)sizeof(typename CellT<R>::type); }

struct SchLayout {
    size_t bar, stage0, stage_bytes, c0, c1, rs, qs, zs, total;
};

template <typename R>
__host__ __device__ inline SchLayout sch_layout(int Tx, int Ty, int ov, int nstage) {
    auto al = [](size_t b) { return (b + 127) & ~(size_t)127; };
    const size_t nc = (size_t)sch_rw(Tx, ov) * sch_rh(Ty, ov);
    SchLayout L;
    L.bar = 0;
    L.c0 = 0;
    L.c1 = al(nc * cell_bytes<R>());
    L.rs = L.c1 + al(nc * cell_bytes<R>());
    L.qs = L.rs + al(3 * (size_t)Tx * Ty * sizeof(R));
    L.stage_bytes = L.qs + al(3 * (size_t)Tx * Ty * sizeof(R));
    L.stage0 = 128;
    L.zs = L.stage0 + (size_t)nstage * L.stage_bytes;
    L.total = L.zs + al(3 * nc * sizeof(R)) + 128;  // + alignment slack
    return L;
}

template <typename R>
__host__ __device__ inline size_t sch_smem_bytes(int Tx, int Ty, int ov, int nstage) {
    return sch_layout<R>(Tx, Ty, ov, nstage).total;
}

// ---------------------------------------------------------------- PTX --
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)tm), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, int x, int y, int z, const void* src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     (uint64_t)tm),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of every committed bulk store have been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed bulk store has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Bounded wait on phase 0 of the staging barrier: returns false after
// `limit` cycles (the caller records the timeout and stops).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, 0)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// Reciprocal of a diagonal pivot.  FP32: the hardware approximation (about 1
// ulp): the preconditioner only has to be one fixed linear operator, which a
// deterministic approximation keeps.  FP64: exact division.
__device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }


__device__ __forceinline__ bool mbar_wait_phase_bounded(uint64_t* bar, unsigned phase, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// ------------------------------------------------------------ cell data --
template <typename R> struct CellView;

template <> struct CellView<float> {
    const uint2* c0;
    const uint2* c1;
    __device__ __forceinline__ static void unpack(uint2 v, float h[3], float& w) {
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
        h[0] = a.x; h[1] = a.y; h[2] = b.x; w = b.y;
    }
    __device__ __forceinline__ void t0(int c, float h[3], float& w) const { unpack(c0[c], h, w); }
    __device__ __forceinline__ void t1(int c, float h[3], float& w) const { unpack(c1[c], h, w); }
};

template <> struct CellView<double> {
    const double4_32a* c0;
    const double4_32a* c1;
    __device__ __forceinline__ void t0(int c, double h[3], double& w) const {
        const double4_32a v = c0[c];
        h[0] = v.x; h[1] = v.y; h[2] = v.z; w = v.w;
    }
    __device__ __forceinline__ void t1(int c, double h[3], double& w) const {
        const double4_32a v = c1[c];
        h[0] = v.x; h[1] = v.y; h[2] = v.z; w = v.w;
    }
};

// Cell records of node (x, y) from the frames and alpha (workspace layouts).
template <typename R>
__device__ __forceinline__ void cell_records(int x, int y, int W, int H, int pitch, R gms, const R* f1, const R* f2,
                                             const R* al, R h0[3], R& wE, R h1[3], R& wN) {
    const R isq24 = R(0.20412414523193151);  // 1/sqrt(24)
    const R third = R(1) / R(3), half = R(0.5);
    const bool vc = (x < W - 1) && (y < H - 1);
    h0[0] = h0[1] = h0[2] = h1[0] = h1[1] = h1[2] = R(0);
    const long long o = (long long)y * pitch + x;
    if (vc) {
        const R a2 = f2[o], b2 = f2[o + 1], c2 = f2[o + pitch + 1], d2 = f2[o + pitch];
        const R a1 = f1[o], b1 = f1[o + 1], c1 = f1[o + pitch + 1], d1 = f1[o + pitch];
        h0[0] = (b2 - a2) * isq24;
        h0[1] = (c2 - b2) * isq24;
        h0[2] = -(a1 + b1 + c1) * third * isq24 * gms;
        h1[0] = (c2 - d2) * isq24;
        h1[1] = (d2 - a2) * isq24;
        h1[2] = -(a1 + d1 + c1) * third * isq24 * gms;
    }
    // edge to (x+1,y): t0 of square (x,y) and t1 of square (x,y-1)
    wE = half * ((vc ? al[2 * o] : R(0)) + ((x < W - 1 && y >= 1) ? al[2 * (o - pitch) + 1] : R(0)));
    // edge to (x,y+1): t1 of square (x,y) and t0 of square (x-1,y)
    wN = half * ((vc ? al[2 * o + 1] : R(0)) + ((x >= 1 && y < H - 1) ? al[2 * (o - 1)] : R(0)));
}

// LDL^T factors of a node's 3x3 diagonal block: 1/d0, l10, l20, 1/d1, l21, 1/d2
template <typename R> struct Blk { R i0, l10, l20, i1, l21, i2; };

template <typename R>
__device__ __forceinline__ Blk<R> ldl3(R D00, R D01, R D02, R D11, R D12, R D22) {
    Blk<R> b;
    b.i0 = rcp(D00);
    b.l10 = D01 * b.i0;
    b.l20 = D02 * b.i0;
    const R d1 = D11 - b.l10 * D01;
    b.i1 = rcp(d1);
    b.l21 = (D12 - b.l20 * D01) * b.i1;
    const R d2 = D22 - b.l20 * D02 - b.l21 * b.l21 * d1;
    b.i2 = rcp(d2);
    return b;
}


// The six elements around node n = cell c (x, y):
//   E1 t0 of (x,y)      others E, NE        E4 t1 of (x-1,y-1) others SW, W
//   E2 t1 of (x,y)      others N, NE        E5 t0 of (x-1,y)   others W, N
//   E3 t0 of (x-1,y-1)  others SW, S        E6 t1 of (x,y-1)   others S, E
// Edge weights: n-E = wE(c), n-N = wN(c), n-W = wE(c-1), n-S = wN(c-RW).
template <typename R>
__device__ __forceinline__ void node_block(const CellView<R>& C, int c, int RW, R lE, R lN, R lW, R lS, Blk<R>& B) {
    R h[6][3], wE, wN, wW, wS, dummy;
    C.t0(c, h[0], wE);
    C.t1(c, h[1], wN);
    C.t0(c - RW - 1, h[2], dummy);
    C.t1(c - RW - 1, h[3], dummy);
    C.t0(c - 1, h[4], wW);
    C.t1(c - RW, h[5], wS);
    R D00 = 0, D01 = 0, D02 = 0, D11 = 0, D12 = 0, D22 = 0;
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        D00 += 2 * h[e][0] * h[e][0]; D01 += 2 * h[e][0] * h[e][1]; D02 += 2 * h[e][0] * h[e][2];
        D11 += 2 * h[e][1] * h[e][1]; D12 += 2 * h[e][1] * h[e][2]; D22 += 2 * h[e][2] * h[e][2];
    }
    const R ws = wE + wN + wW + wS;
    B = ldl3<R>(D00 + ws, D01, D02, D11 + ws, D12, D22 + (lE + lN + lW + lS));
}

// lambda weight of a leg: 1/2 lambda per triangle on it (legs: 2-bit counts
// E, N, W, S); away from the image border every leg has two
template <typename R>
__device__ __forceinline__ R lam_edges(unsigned legs, R hl, R zE2, R zN2, R zW2, R zS2) {
    if (legs == 0xAAu) return (hl + hl) * ((zE2 + zN2) + (zW2 + zS2));
    return hl * (R(legs & 3u) * zE2 + R((legs >> 2) & 3u) * zN2 + R((legs >> 4) & 3u) * zW2 + R(legs >> 6) * zS2);
}

template <typename R>
__device__ __forceinline__ void block_solve(const Blk<R>& B, R b0, R b1, R b2, R& x0, R& x1, R& x2) {
    const R y1 = b1 - B.l10 * b0, y2 = b2 - B.l20 * b0 - B.l21 * y1;
    x2 = y2 * B.i2;
    x1 = y1 * B.i1 - B.l21 * x2;
    x0 = b0 * B.i0 - B.l10 * x1 - B.l20 * x2;
}

// z_n <- z_n + omega (x - z_n); FRESH: first visit of the colour in this
// subdomain, z_n is still zero (its shared-memory slot holds another item's data)
template <typename R, bool FRESH>
__device__ __forceinline__ void relax(const R* Z, int zplane, int c, R om, R& x0, R& x1, R& x2) {
    if (FRESH) {
        x0 *= om;
        x1 *= om;
        x2 *= om;
    } else {
        const R o0 = Z[c], o1 = Z[c + zplane], o2 = Z[c + 2 * zplane];
        x0 = o0 + om * (x0 - o0);
        x1 = o1 + om * (x1 - o1);
        x2 = o2 + om * (x2 - o2);
    }
}

template <typename R, bool FRESH = false>
__device__ __forceinline__ void node_sweep(const CellView<R>& C, R* __restrict__ Z, int zplane, int c, int RW,
                                           unsigned legs, R hl, R om, const Blk<R>& B, R b0, R b1, R b2, R& x0,
                                           R& x1, R& x2) {
    const R* z0 = Z;
    const R* z1 = Z + zplane;
    const R* z2 = Z + 2 * zplane;
    const int iE = c + 1, iW = c - 1, iN = c + RW, iS = c - RW, iNE = c + RW + 1, iSW = c - RW - 1;
    const R zE0 = z0[iE], zE1 = z1[iE], zE2 = z2[iE];
    const R zW0 = z0[iW], zW1 = z1[iW], zW2 = z2[iW];
    const R zN0 = z0[iN], zN1 = z1[iN], zN2 = z2[iN];
    const R zS0 = z0[iS], zS1 = z1[iS], zS2 = z2[iS];
    const R zNE0 = z0[iNE], zNE1 = z1[iNE], zNE2 = z2[iNE];
    const R zSW0 = z0[iSW], zSW1 = z1[iSW], zSW2 = z2[iSW];
    R h[3] = {R(0), R(0), R(0)}, wE, wN, wW, wS, dummy;
    auto elem = [&](R s0, R s1, R s2) {
        const R s = h[0] * s0 + h[1] * s1 + h[2] * s2;
        b0 -= s * h[0];
        b1 -= s * h[1];
        b2 -= s * h[2];
    };
    C.t0(c, h, wE);             elem(zE0 + zNE0, zE1 + zNE1, zE2 + zNE2);  // E1
    C.t1(c, h, wN);             elem(zN0 + zNE0, zN1 + zNE1, zN2 + zNE2);  // E2
    C.t0(c - RW - 1, h, dummy); elem(zSW0 + zS0, zSW1 + zS1, zSW2 + zS2);  // E3
    C.t1(c - RW - 1, h, dummy); elem(zSW0 + zW0, zSW1 + zW1, zSW2 + zW2);  // E4
    C.t0(c - 1, h, wW);         elem(zW0 + zN0, zW1 + zN1, zW2 + zN2);     // E5
    C.t1(c - RW, h, wS);        elem(zS0 + zE0, zS1 + zE1, zS2 + zE2);     // E6
    b0 += wE * zE0 + wN * zN0 + wW * zW0 + wS * zS0;
    b1 += wE * zE1 + wN * zN1 + wW * zW1 + wS * zS1;
    b2 += lam_edges(legs, hl, zE2, zN2, zW2, zS2);
    block_solve(B, b0, b1, b2, x0, x1, x2);
    if (om != R(1)) relax<R, FRESH>(Z, zplane, c, om, x0, x1, x2);
    Z[c] = x0;
    Z[c + zplane] = x1;
    Z[c + 2 * zplane] = x2;
}

// The first colour-1 update of a sweep sequence that starts from z = 0 and
// a colour-0 block-Jacobi step: the colour-2 neighbours (E, N, SW) are still
// zero, so only the W, S and NE values enter.
template <typename R>
__device__ __forceinline__ void node_sweep_first1(const CellView<R>& C, R* __restrict__ Z, int zplane, int c, int RW,
                                                  unsigned legs, R hl, R om, const Blk<R>& B, R b0, R b1, R b2) {
    const R* z0 = Z;
    const R* z1 = Z + zplane;
    const R* z2 = Z + 2 * zplane;
    const int iW = c - 1, iS = c - RW, iNE = c + RW + 1;
    const R zW0 = z0[iW], zW1 = z1[iW], zW2 = z2[iW];
    const R zS0 = z0[iS], zS1 = z1[iS], zS2 = z2[iS];
    const R zNE0 = z0[iNE], zNE1 = z1[iNE], zNE2 = z2[iNE];
    R h[3] = {R(0), R(0), R(0)}, wW, wS, dummy;
    auto elem = [&](R s0, R s1, R s2) {
        const R s = h[0] * s0 + h[1] * s1 + h[2] * s2;
        b0 -= s * h[0];
        b1 -= s * h[1];
        b2 -= s * h[2];
    };
    C.t0(c, h, dummy);          elem(zNE0, zNE1, zNE2);  // E1
    C.t1(c, h, dummy);          elem(zNE0, zNE1, zNE2);  // E2
    C.t0(c - RW - 1, h, dummy); elem(zS0, zS1, zS2);     // E3
    C.t1(c - RW - 1, h, dummy); elem(zW0, zW1, zW2);     // E4
    C.t0(c - 1, h, wW);         elem(zW0, zW1, zW2);     // E5
    C.t1(c - RW, h, wS);        elem(zS0, zS1, zS2);     // E6
    b0 += wW * zW0 + wS * zS0;
    b1 += wW * zW1 + wS * zS1;
    const R z = R(0);
    b2 += lam_edges(legs, hl, z, z, zW2, zS2);
    R x0, x1, x2;
    block_solve(B, b0, b1, b2, x0, x1, x2);
    if (om != R(1)) relax<R, true>(Z, zplane, c, om, x0, x1, x2);
    Z[c] = x0;
    Z[c + zplane] = x1;
    Z[c + 2 * zplane] = x2;
}

__device__ __forceinline__ double block_sum_rt(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (l < nw) ? sh[l] : 0.0;
        s = warp_sum(s);
    }
    return s;
}

__device__ __forceinline__ double ordered_sum_rt(const double* p, int n, int stride, double* sh) {
    return block_sum_rt(strided_sum8(p, n, stride, threadIdx.x, blockDim.x), sh);
}


// CG scalars of one pair after its preconditioned residual is complete:
// t_rr = r.r, t_rz = r.z over the pair; first = start of a pass.
__device__ __forceinline__ void precond_finalize(PairScalars* sp, double t_rr, double t_rz, int first) {
    if (first) {
        sp->rz = t_rz;
        sp->rr = t_rr;
        sp->beta = 0.0;
        if (!isfinite(t_rr) || !isfinite(t_rz)) { sp->status = 6; sp->done = 1; }
        else if (t_rr <= sp->tol2 || t_rr == 0.0) { sp->done = 1; }
        else if (!(t_rz > 0.0)) { sp->status = 6; sp->done = 1; }
    } else {
        sp->beta = t_rz / sp->rz;
        sp->rz = t_rz;
        sp->rr = t_rr;
        sp->it += 1;
        sp->it_total += 1;
        if (!isfinite(t_rr) || !isfinite(t_rz)) { sp->status = 6; sp->done = 1; }
        else if (t_rr <= sp->tol2) { sp->done = 1; }
        else if (!(t_rz > 0.0)) { sp->status = 6; sp->done = 1; }
        else if (sp->it >= sp->max_it) { sp->status = 5; sp->done = 1; }
    }
}

// Largest CTA the host may build a node table for (registers: the owned
// nodes' blocks and right-hand sides live in registers).
__host__ __device__ constexpr int sch_max_threads(bool fp64) { return fp64 ? 384 : 384; }

// Per-node sweep state kept in registers by the owning thread.
template <typename R> struct NodeState {
    int c;            // cell index (low 24 bits; -1: no node) | triangles on the E,N,W,S legs (2 bits each)
    R b0, b1, b2;     // right-hand side
    Blk<R> B;         // LDL^T factors of the diagonal block
};

// Output of the last visit of a colour: the owned part of the local
// solution into the dense tile that is bulk-stored, and the partial r.z.
template <typename R>
struct ZOut {
    R* zo;       // [3][Ty][Tx] tile of z
    int Tx, plane, tw, th, ov, cpad, RW;
    R rz;
    int* err;
    __device__ __forceinline__ void emit(const NodeState<R>& n, R x0, R x1, R x2) {
        const int c = n.c & 0xffffff;
        const int row = c / RW;                      // lj + 1
        const int ox = c - row * RW - cpad, oy = row - 1 - ov;  // position in the owned tile
        if (ox < 0 || ox >= tw || oy < 0 || oy >= th) return;
        if (!OF_CHECK(err, oy * Tx + ox, plane)) return;
        const int si = oy * Tx + ox;
        zo[si] = x0;
        zo[si + plane] = x1;
        zo[si + 2 * plane] = x2;
        rz += n.b0 * x0 + n.b1 * x1 + n.b2 * x2;
    }
};

template <typename R, bool FRESH = false, bool LAST = false>
__device__ __forceinline__ void node_step(const CellView<R>& C, R* Zs, int nc, int RW, R hl, R om,
                                          const NodeState<R>& n, ZOut<R>& out) {
    if (n.c == -1) return;
    R x0, x1, x2;
    node_sweep<R, FRESH>(C, Zs, nc, n.c & 0xffffff, RW, (unsigned)n.c >> 24, hl, om, n.B, n.b0, n.b1, n.b2, x0, x1,
                         x2);
    if (LAST) out.emit(n, x0, x1, x2);
}
template <typename R>
__device__ __forceinline__ void node_step_first1(const CellView<R>& C, R* Zs, int nc, int RW, R hl, R om,
                                                 const NodeState<R>& n) {
    if (n.c == -1) return;
    node_sweep_first1<R>(C, Zs, nc, n.c & 0xffffff, RW, (unsigned)n.c >> 24, hl, om, n.B, n.b0, n.b1, n.b2);
}

// Block Jacobi: z = D^{-1} r, no neighbour terms.
template <typename R>
__device__ __forceinline__ void node_jacobi(R* Zs, int nc, const NodeState<R>& n, R om = R(1)) {
    if (n.c == -1) return;
    const int c = n.c & 0xffffff;
    R x0, x1, x2;
    block_solve(n.B, n.b0, n.b1, n.b2, x0, x1, x2);
    if (om != R(1)) {
        x0 *= om;
        x1 *= om;
        x2 *= om;
    }
    Zs[c] = x0;
    Zs[c + nc] = x1;
    Zs[c + 2 * nc] = x2;
}

template <typename R, int NPT, int TXC, int TYC, int OVC>
__global__ void __launch_bounds__(sch_max_threads(sizeof(R) == 8), 1) k_schwarz(const SchwarzParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ double sh_red[32];
    __shared__ int sh_last, sh_fail;
    const int NT = blockDim.x;
    // compile-time for the tuned tile shapes (TXC > 0), runtime otherwise
    const int Tx = TXC ? TXC : P.Tx, Ty = TXC ? TYC : P.Ty, ov = TXC ? OVC : P.ov;
    const int RW = sch_rw(Tx, ov);
    const int RH = sch_rh(Ty, ov);
    const int nc = RW * RH;
    const int cpad = sch_cpad(ov);
    const int nstage = P.nstage;
    const SchLayout L = sch_layout<R>(Tx, Ty, ov, nstage);
    unsigned char* base = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bar);
    R* Zs = reinterpret_cast<R*>(base + L.zs);
    const unsigned box_rq = (unsigned)(3 * (size_t)Tx * Ty * sizeof(R));
    const unsigned box_c = (unsigned)(nc * cell_bytes<R>());

    if (threadIdx.x == 0) {
        sh_fail = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    // the ring around the extended tile is never written: the Dirichlet zeros
    // of every item.  Inside the extended tile every position is written by its
    // owner before it is read (zeros where the tile is clipped by the image).
    for (int i = threadIdx.x; i < 3 * nc; i += NT) Zs[i] = R(0);
    __syncthreads();

    // a work item is processed unless its pair has finished (a pair's flag is
    // only set after all of its items have been processed in this launch)
    auto issue = [&](const int4 ti, int s) {
        const CUtensorMap* tm = P.tmaps + (size_t)ti.x * TM_PER_PAIR;
        const int x0 = ti.y * Tx, y0 = ti.z * Ty;
        const bool need_q = !P.first && !P.apply_only;
        unsigned char* st = base + L.stage0 + (size_t)s * L.stage_bytes;
        // the stores that read this stage last time are done reading; order this
        // stage's earlier generic-proxy accesses before the async-proxy writes
        bulk_wait_read();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bars[s], 2 * box_c + box_rq + (need_q ? box_rq : 0u) + (unsigned)P.tx_extra);
        const int cx = (x0 - cpad) * CellT<R>::units, cy = y0 - ov - 1;
        tma_load_2d(st + L.c0, tm + TM_C0, cx, cy, &bars[s]);
        tma_load_2d(st + L.c1, tm + TM_C1, cx, cy, &bars[s]);
        tma_load_3d(st + L.rs, tm + TM_R, x0, y0, 0, &bars[s]);
        if (need_q) tma_load_3d(st + L.qs, tm + TM_Q, x0, y0, 0, &bars[s]);
    };
    const int G = gridDim.x;
    // A pair's done flag only changes in the last CTA, after every item of
    // the launch: read the first 32 once (a register mask), so that skipping
    // finished pairs costs no dependent global load per item.
    unsigned done_mask = 0u;
    if (!P.apply_only && P.npairs <= 32) {
        const int l = threadIdx.x & 31;
        done_mask = __ballot_sync(0xffffffffu, l < P.npairs && P.sc[l].done != 0);
    }
    auto pair_done = [&](int pair) -> bool {
        if (P.apply_only) return false;
        if (P.npairs <= 32) return (done_mask >> pair) & 1u;
        return P.sc[pair].done != 0;
    };
    // next active item at or after t (slow path: loads until an active one)
    auto advance = [&](int t, int4& ti) {
        while (t < P.ntiles) {
            ti = P.tiles[t];
            if (!pair_done(ti.x)) return t;
            t += G;
        }
        return t;
    };

    // this thread's nodes of the (unclipped) extended tile, per colour
    uint32_t tab[3][NPT];
#pragma unroll
    for (int col = 0; col < 3; ++col)
#pragma unroll
        for (int k = 0; k < NPT; ++k) tab[col][k] = P.ntab[(col * NPT + k) * NT + threadIdx.x];

    int4 ti = make_int4(0, 0, 0, 0), tin = make_int4(0, 0, 0, 0);
    int t = advance(blockIdx.x, ti);
    int tn = (t < P.ntiles) ? advance(t + G, tin) : P.ntiles;
    if (t < P.ntiles && threadIdx.x == 0) issue(ti, 0);
    unsigned phase[2] = {0u, 0u};
    int s = 0;
    for (; t < P.ntiles;) {
        // software pipelining: the item after next is fetched now and used one
        // iteration later, so its descriptor loads overlap this item's work
        const int tc = tn + G;
        int4 tic = make_int4(0, 0, 0, 0);
        if (tn < P.ntiles && tc < P.ntiles) tic = P.tiles[tc];  // used at the end of this item

        if (threadIdx.x == 0 && !mbar_wait_phase_bounded(&bars[s], phase[s], P.spin_limit)) {
            sh_fail = 1;
            atomicOr(P.err, 1);
        }
        __syncthreads();
        if (sh_fail) {
            // give the copies in flight a last chance to land, then stop
            // processing (the CTA still arrives below, so the launch ends)
            // (the next item's copies are only issued after the setup below)
            if (threadIdx.x == 0) mbar_wait_phase_bounded(&bars[s], phase[s], P.spin_limit);
            break;
        }
        if (!mbar_wait_phase_bounded(&bars[s], phase[s], P.spin_limit)) atomicOr(P.err, 1);
        phase[s] ^= 1u;

        unsigned char* st = base + L.stage0 + (size_t)s * L.stage_bytes;
        CellView<R> C;
        C.c0 = reinterpret_cast<const typename CellT<R>::type*>(st + L.c0);
        C.c1 = reinterpret_cast<const typename CellT<R>::type*>(st + L.c1);
        R* Rs = reinterpret_cast<R*>(st + L.rs);
        const R* Qs = reinterpret_cast<const R*>(st + L.qs);

        const int pair = ti.x;
        const PairDesc pd = P.pairs[pair];
        const int W = pd.W, H = pd.H;
        const int x0 = ti.y * Tx, y0 = ti.z * Ty;
        const int tw = min(Tx, W - x0), th = min(Ty, H - y0);
        const int ex0 = max(x0 - ov, 0), ex1 = min(x0 + tw + ov, W);
        const int ey0 = max(y0 - ov, 0), ey1 = min(y0 + th + ov, H);
        const bool need_q = !P.first && !P.apply_only;

        // ---- owned nodes: diagonal blocks, right-hand sides, r <- r - a q
        const R a = need_q ? (R)P.sc[pair].a : R(0);
        const R hl = R(0.5) * (R)P.lam;
        const R om = (R)P.omega;
        R rr = R(0);  // partial r.r of the owned nodes
        NodeState<R> ns[3][NPT];
#pragma unroll
        for (int col = 0; col < 3; ++col) {
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                const uint32_t e = tab[col][k];
                NodeState<R>& n = ns[col][k];
                n.c = -1;
                n.b0 = n.b1 = n.b2 = R(0);
                n.B = Blk<R>{R(0), R(0), R(0), R(0), R(0), R(0)};
                if (e == 0xffffffffu) continue;
                const int li = (int)(e & 0xffffu), lj = (int)(e >> 16);
                const int gx = x0 - ov + li, gy = y0 - ov + lj;
                const int c = (lj + 1) * RW + (li + cpad - ov);
                // every access of the node's sweeps lies in [c - RW - 1, c + RW + 1] of
                // each z plane and of the record planes
                if (!OF_CHECK(P.err, c - RW - 1, nc) || !OF_CHECK(P.err, c + RW + 1, nc)) continue;
                if (gx < ex0 || gx >= ex1 || gy < ey0 || gy >= ey1) {
                    Zs[c] = R(0);
                    Zs[c + nc] = R(0);
                    Zs[c + 2 * nc] = R(0);
                    continue;
                }
                // existing triangles on the four legs (the lambda weight is 1/2 lambda each)
                const int vc = (gx < W - 1 && gy < H - 1), vsw = (gx >= 1 && gy >= 1);
                const int vw = (gx >= 1 && gy < H - 1), vs = (gx < W - 1 && gy >= 1);
                const int nE = vc + vs, nN = vc + vw, nW = vsw + vw, nS = vsw + vs;
                n.c = c | (nE << 24) | (nN << 26) | (nW << 28) | (nS << 30);
                node_block<R>(C, c, RW, hl * R(nE), hl * R(nN), hl * R(nW), hl * R(nS), n.B);
                if (gx >= x0 && gx < x0 + tw && gy >= y0 && gy < y0 + th &&
                    OF_CHECK(P.err, (gy - y0) * Tx + (gx - x0), Tx * Ty)) {
                    const int si = (gy - y0) * Tx + (gx - x0);
                    R v0 = Rs[si], v1 = Rs[si + Tx * Ty], v2 = Rs[si + 2 * Tx * Ty];
                    if (need_q) {
                        v0 -= a * Qs[si];
                        v1 -= a * Qs[si + Tx * Ty];
                        v2 -= a * Qs[si + 2 * Tx * Ty];
                        Rs[si] = v0;
                        Rs[si + Tx * Ty] = v1;
                        Rs[si + 2 * Tx * Ty] = v2;
                    }
                    n.b0 = v0;
                    n.b1 = v1;
                    n.b2 = v2;
                    rr += v0 * v0 + v1 * v1 + v2 * v2;
                }
                // the first colour step from z = 0 is (relaxed) block Jacobi on colour 0
                if (col == 0) node_jacobi<R>(Zs, nc, n, P.sweeps > 0 ? om : R(1));
            }
        }
        __syncthreads();
        // the next active item of this CTA goes into the other stage (the bulk
        // stores that read that stage were issued an item ago and are done by now)
        if (nstage == 2 && tn < P.ntiles && threadIdx.x == 0) issue(tin, s ^ 1);

        // ---- sweeps (colour order 0,1,2,1,0,1,2,1,0,...; sweeps = 0: block Jacobi).
        // The last visit of each colour also writes the owned z into the q
        // buffer of this stage (q was consumed in the setup) for the bulk
        // store, and accumulates r.z.
        ZOut<R> zout;
        zout.zo = reinterpret_cast<R*>(st + L.qs);
        zout.Tx = Tx;
        zout.plane = Tx * Ty;
        zout.tw = tw;
        zout.th = th;
        zout.ov = ov;
        zout.cpad = cpad;
        zout.RW = RW;
        zout.rz = R(0);
        zout.err = P.err;
#define OF_STEP(col, FRESH, LAST)                                                 \
    {                                                                             \
        _Pragma("unroll") for (int k = 0; k < NPT; ++k)                           \
            node_step<R, FRESH, LAST>(C, Zs, nc, RW, hl, om, ns[col][k], zout);   \
        __syncthreads();                                                          \
    }
        if (P.sweeps == 0) {
#pragma unroll
            for (int col = 1; col < 3; ++col)
#pragma unroll
                for (int k = 0; k < NPT; ++k) node_jacobi<R>(Zs, nc, ns[col][k]);
            __syncthreads();
#pragma unroll
            for (int col = 0; col < 3; ++col)
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    const NodeState<R>& n = ns[col][k];
                    if (n.c == -1) continue;
                    const int c = n.c & 0xffffff;
                    zout.emit(n, Zs[c], Zs[c + nc], Zs[c + 2 * nc]);
                }
        } else {
            // colour 0 of the first sweep was the Jacobi step above; colours 1
            // and 2 start from zero on their first visit
#pragma unroll
            for (int k = 0; k < NPT; ++k) node_step_first1<R>(C, Zs, nc, RW, hl, om, ns[1][k]);
            __syncthreads();
            if (P.sweeps == 1) {
                OF_STEP(2, true, true)
                OF_STEP(1, false, true)
                OF_STEP(0, false, true)
            } else {
                OF_STEP(2, true, false)
                OF_STEP(1, false, false)
                for (int sw = 2; sw < P.sweeps; ++sw) {
                    OF_STEP(0, false, false)
                    OF_STEP(1, false, false)
                    OF_STEP(2, false, false)
                    OF_STEP(1, false, false)
                }
                OF_STEP(0, false, false)
                OF_STEP(1, false, false)
                OF_STEP(2, false, true)
                OF_STEP(1, false, true)
                OF_STEP(0, false, true)
            }
        }
#undef OF_STEP

        R* Zo = zout.zo;
        const R rz = zout.rz;
        const float wrr = warp_sum((float)rr), wrz = warp_sum((float)rz);
        if ((threadIdx.x & 31) == 0) {
            sh_red[threadIdx.x >> 5] = (double)wrr;
            sh_red[16 + (threadIdx.x >> 5)] = (double)wrz;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // bulk stores of the owned tile: z from the q buffer, updated r
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const CUtensorMap* tm = P.tmaps + (size_t)pair * TM_PER_PAIR;
            tma_store_3d(tm + TM_Z, x0, y0, 0, Zo);
            if (need_q) tma_store_3d(tm + TM_R, x0, y0, 0, Rs);
            bulk_commit();
        }
        if (!P.apply_only && threadIdx.x < 32) {
            // the item's partials: warp sums of the CTA in a fixed order
            const int l = threadIdx.x;
            const bool w = l < (NT >> 5);
            const double a2 = warp_sum(w ? sh_red[l] : 0.0), b2 = warp_sum(w ? sh_red[16 + l] : 0.0);
            if (l == 0) {
                P.partial[2 * (long long)ti.w] = a2;
                P.partial[2 * (long long)ti.w + 1] = b2;
            }
        }
        __syncthreads();  // z and the partial slots are free for the next item
        t = tn;
        ti = tin;
        tn = tc;
        tin = tic;
        if (tn < P.ntiles && pair_done(tin.x)) tn = advance(tn + G, tin);  // the fetched item's pair has finished
        if (nstage == 2) s ^= 1;
        else if (t < P.ntiles && threadIdx.x == 0) issue(ti, 0);
    }
    if (threadIdx.x == 0) bulk_wait_all();  // the last stores have landed before the CTA leaves
    if (P.apply_only || P.defer) return;    // defer: the coarse correction finishes the scalars
    // one arrival per CTA; the last CTA reduces the items of every pair that
    // took part, in item order (deterministic), and updates its scalars
    if (!arrive_last(P.counter, gridDim.x, &sh_last)) return;
    for (int pi = 0; pi < P.npairs; ++pi) {
        PairScalars* sp = P.sc + pi;
        if (sp->done) continue;  // finished before this launch: nothing of it ran
        const PairDesc pd = P.pairs[pi];
        const int ntp = pd.tiles_x * pd.tiles_y;
        const double t_rr = ordered_sum_rt(P.partial + 2 * (long long)pd.tile0, ntp, 2, sh_red);
        const double t_rz = ordered_sum_rt(P.partial + 2 * (long long)pd.tile0 + 1, ntp, 2, sh_red);
        if (threadIdx.x == 0) precond_finalize(sp, t_rr, t_rz, P.first);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (P.use_cond) {
            // keep looping while a pair is still iterating and no wait ran out
            int more = 0;
            for (int pi = 0; pi < P.npairs; ++pi) more |= !P.sc[pi].done;
            if (*(volatile int*)P.err) more = 0;
            cudaGraphSetConditional(P.cond, more ? 1u : 0u);
        }
        __threadfence();
        *P.counter = 0u;
    }
}

// Cell records for every node of every pair (once per solve).
template <typename R>
__global__ void k_cells(const PairDesc* pairs, int pair, R gms, const R* __restrict__ f1a, const R* __restrict__ f2a,
                        const R* __restrict__ ala, typename CellT<R>::type* __restrict__ c0a,
                        typename CellT<R>::type* __restrict__ c1a) {
    const PairDesc pd = pairs[pair];
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= pd.W) return;
    R h0[3], h1[3], wE, wN;
    cell_records<R>(x, y, pd.W, pd.H, pd.pitch, gms, f1a + pd.frame_off, f2a + pd.frame_off, ala + 2 * pd.frame_off, h0,
                    wE, h1, wN);
    const long long o = pd.frame_off + (long long)y * pd.pitch + x;
    if constexpr (sizeof(R) == 4) {
        const __half2 a = __floats2half2_rn(h0[0], h0[1]), b = __floats2half2_rn(h0[2], wE);
        const __half2 c = __floats2half2_rn(h1[0], h1[1]), d = __floats2half2_rn(h1[2], wN);
        c0a[o] = make_uint2(*reinterpret_cast<const unsigned*>(&a), *reinterpret_cast<const unsigned*>(&b));
        c1a[o] = make_uint2(*reinterpret_cast<const unsigned*>(&c), *reinterpret_cast<const unsigned*>(&d));
    } else {
        c0a[o] = make_double4_32a(h0[0], h0[1], h0[2], wE);
        c1a[o] = make_double4_32a(h1[0], h1[1], h1[2], wN);
    }
}

}  // namespace ofk
