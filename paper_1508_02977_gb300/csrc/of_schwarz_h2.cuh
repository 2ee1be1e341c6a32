// Overlapping Schwarz preconditioner, FP16 paired form (mixed path).
//
// The same operator as k_schwarz (of_schwarz.cuh): symmetric restricted
// Schwarz on extended tiles, local solves by s symmetric 3-colour block SOR
// sweeps from zero (Section 3.2, Eq. schwarz), but the sweeps run in packed
// half-precision arithmetic on two nodes at once.  The extended tile of
// Ex x Ey nodes is cut into a top half (rows 0 .. HP-1) and a bottom half
// (rows HP .. 2HP-1), HP = Ey / 2 a multiple of 3, so that node (i, j) and
// node (i, j + HP) have the same colour; they share one half2 lane pair in
// every shared-memory word (lane A: top, lane B: bottom) and one thread
// updates both with the same instructions.  One 32-bit load then serves two
// node updates, the element records need no conversion, and every FMA works
// on two nodes.
//
// Range: the local solve is linear, so it is run on the scaled right-hand
// side b / m, m = max over the tile of |D_n^{-1} b_n| (the first Jacobi
// step), which keeps the iterates of order one, and the result is scaled
// back in FP32.  The residual update r <- r - a q, the diagonal blocks and
// their LDL^T factors are formed in FP32 (the factors are then rounded to
// FP16), and r.z is accumulated in FP32 from the FP32 residual, so only the
// sweep arithmetic is in half precision.
//
// Seam: the top half's last row (HP-1) and the bottom half's first row (HP)
// are stencil neighbours.  Their values are also kept in two ghost rows of
// the paired array: paired row -1, lane B holds node row HP-1 (the south
// neighbour of lane B's paired row 0), paired row HP, lane A holds node row
// HP (the north neighbour of lane A's paired row HP-1); the other lanes of
// those rows are the Dirichlet ring (zero).  A node on a seam row writes its
// ghost in the same colour step as itself, so the colour schedule that makes
// the sweeps race-free covers the ghosts as well.
#pragma once
#include <cuda_fp16.h>

#include "of_df.cuh"
#include "of_schwarz.cuh"

namespace ofk {

// paired element record of one square: (h0, h1, h2, w) of the top node's
// square (lane A) and of the square HP rows below it (lane B)
struct __align__(16) RecH2 {
    __half2 h0, h1, h2, w;
};

struct H2Layout {
    size_t bar, stage0, stage_bytes, p0, p1, rs, qs, zs, total;
};

__host__ __device__ inline int h2_hp(int Ty, int ov) { return (Ty + 2 * ov) / 2; }

// Records of the window: RW x (HP + 1) per triangle family (ext rows -1 .. HP-1
// in lane A); z: 3 planes of RW x (HP + 2) half2 (paired rows -1 .. HP).
__host__ __device__ inline H2Layout h2_layout(int Tx, int Ty, int ov, int nstage) {
    auto al = [](size_t b) { return (b + 127) & ~(size_t)127; };
    const int HP = h2_hp(Ty, ov), RW = sch_rw(Tx, ov);
    const size_t nr = (size_t)RW * (HP + 1), nz = (size_t)RW * (HP + 2);
    H2Layout L;
    L.bar = 0;
    L.p0 = 0;
    L.p1 = al(nr * sizeof(RecH2));
    L.rs = L.p1 + al(nr * sizeof(RecH2));
    L.qs = L.rs + al(3 * (size_t)Tx * Ty * sizeof(float));
    L.stage_bytes = L.qs + al(3 * (size_t)Tx * Ty * sizeof(float));
    L.stage0 = 128;
    L.zs = L.stage0 + (size_t)nstage * L.stage_bytes;
    L.total = L.zs + al(3 * nz * sizeof(__half2)) + 128;
    return L;
}

__host__ __device__ inline size_t h2_smem_bytes(int Tx, int Ty, int ov, int nstage) {
    return h2_layout(Tx, Ty, ov, nstage).total;
}

// Whether a tile shape can use the paired form: an even extended height whose
// half is a multiple of 3 (the two lanes of a word then have one colour).
__host__ __device__ inline bool h2_shape_ok(int Ty, int ov) {
    const int Ey = Ty + 2 * ov;
    return Ey % 2 == 0 && (Ey / 2) % 3 == 0;
}

__device__ __forceinline__ float h_lo(__half2 v) { return __low2float(v); }
__device__ __forceinline__ float h_hi(__half2 v) { return __high2float(v); }
__device__ __forceinline__ float h_lane(__half2 v, int L) { return L ? __high2float(v) : __low2float(v); }

// LDL^T factors of a pair of 3x3 diagonal blocks (as Blk<float>, lane-packed)
struct BlkH2 {
    __half2 i0, l10, l20, i1, l21, i2;
};

__device__ __forceinline__ void block_solve_h2(const BlkH2& B, __half2 b0, __half2 b1, __half2 b2, __half2& x0,
                                               __half2& x1, __half2& x2) {
    const __half2 y1 = __hfma2(__hneg2(B.l10), b0, b1);
    const __half2 y2 = __hfma2(__hneg2(B.l21), y1, __hfma2(__hneg2(B.l20), b0, b2));
    x2 = __hmul2(y2, B.i2);
    x1 = __hfma2(__hneg2(B.l21), x2, __hmul2(y1, B.i1));
    x0 = __hfma2(__hneg2(B.l20), x2, __hfma2(__hneg2(B.l10), x1, __hmul2(b0, B.i0)));
}

// b <- b - h (h . (za + zb)) for one element, both lanes
__device__ __forceinline__ void elem_h2(const RecH2& r, __half2 za0, __half2 za1, __half2 za2, __half2 zb0,
                                        __half2 zb1, __half2 zb2, __half2& b0, __half2& b1, __half2& b2) {
    const __half2 s0 = __hadd2(za0, zb0), s1 = __hadd2(za1, zb1), s2 = __hadd2(za2, zb2);
    const __half2 s = __hfma2(r.h2, s2, __hfma2(r.h1, s1, __hmul2(r.h0, s0)));
    const __half2 ns = __hneg2(s);
    b0 = __hfma2(ns, r.h0, b0);
    b1 = __hfma2(ns, r.h1, b1);
    b2 = __hfma2(ns, r.h2, b2);
}

// Per-thread state of one node pair (one colour): the cell index (-1: no
// pair), the scaled right-hand sides, the factors, the current values, and
// the lambda weights of the E/W and N/S legs (1/2 lambda per triangle on the
// leg: lambda on interior legs, lambda/2 along the image border).
struct PairState {
    int c;
    int seam;  // 1: paired row HP-1 (writes the lane-A ghost), 2: paired row 0 (lane-B ghost)
    __half2 b0, b1, b2;
    BlkH2 B;
    __half2 z0, z1, z2;
    __half2 lew, lns;
};

// LDL^T factors of the two diagonal blocks of a node pair and the lambda
// weights of its legs, both lanes, in FP32 (zero for a clipped lane).
struct FacF2 {
    float2 i0, l10, l20, i1, l21, i2, lew, lns;
};

// The factors of the node pair at (gx, gyA) / (gx, gyB) from its six paired
// records: D = sum_K 2 h_K h_K^T + the alpha edge weights on the (u1, u2)
// diagonal + the lambda legs on the m diagonal, both lanes in packed FP32
// arithmetic; vA, vB: the lane's node lies in the extended tile.
__device__ __forceinline__ FacF2 pair_factors(const RecH2 (&rec)[6], int gx, int gyA, int gyB, bool vA, bool vB,
                                              int W, int H, float hl) {
    const float2 zero2 = make_float2(0.f, 0.f);
    float2 S00 = zero2, S01 = zero2, S02 = zero2, S11 = zero2, S12 = zero2, S22 = zero2;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float2 a0 = __half22float2(rec[k].h0), a1 = __half22float2(rec[k].h1), a2 = __half22float2(rec[k].h2);
        S00 = __ffma2_rn(a0, a0, S00);
        S01 = __ffma2_rn(a0, a1, S01);
        S02 = __ffma2_rn(a0, a2, S02);
        S11 = __ffma2_rn(a1, a1, S11);
        S12 = __ffma2_rn(a1, a2, S12);
        S22 = __ffma2_rn(a2, a2, S22);
    }
    // alpha edge weights E, N, W, S: w of E1, E2, E5, E6
    const float2 ws = __fadd2_rn(__fadd2_rn(__half22float2(rec[0].w), __half22float2(rec[1].w)),
                                 __fadd2_rn(__half22float2(rec[4].w), __half22float2(rec[5].w)));
    // lambda legs: 1/2 lambda per triangle on each of the four legs
    auto legs = [&](int gy) {
        const int vc = (gx < W - 1 && gy < H - 1), vsw = (gx >= 1 && gy >= 1);
        const int vw = (gx >= 1 && gy < H - 1), vs = (gx < W - 1 && gy >= 1);
        return (float)((vc + vs) + (vc + vw) + (vsw + vw) + (vsw + vs));
    };
    const float2 two = make_float2(2.f, 2.f);
    const float2 D00 = __ffma2_rn(two, S00, ws), D01 = __fmul2_rn(two, S01), D02 = __fmul2_rn(two, S02),
                 D11 = __ffma2_rn(two, S11, ws), D12 = __fmul2_rn(two, S12);
    const float2 D22 = __ffma2_rn(two, S22, make_float2(hl * legs(gyA), hl * legs(gyB)));
    auto neg = [](float2 v) { return make_float2(-v.x, -v.y); };
    const float2 i0 = make_float2(rcp(D00.x), rcp(D00.y));
    const float2 l10 = __fmul2_rn(D01, i0), l20 = __fmul2_rn(D02, i0);
    const float2 d1 = __ffma2_rn(neg(l10), D01, D11);
    const float2 i1 = make_float2(rcp(d1.x), rcp(d1.y));
    const float2 l21 = __fmul2_rn(__ffma2_rn(neg(l20), D01, D12), i1);
    const float2 d2 = __ffma2_rn(neg(l21), __fmul2_rn(l21, d1), __ffma2_rn(neg(l20), D02, D22));
    const float2 i2 = make_float2(rcp(d2.x), rcp(d2.y));
    auto mask = [&](float2 v) { return make_float2(vA ? v.x : 0.f, vB ? v.y : 0.f); };
    FacF2 f;
    f.i0 = mask(i0);
    f.l10 = mask(l10);
    f.l20 = mask(l20);
    f.i1 = mask(i1);
    f.l21 = mask(l21);
    f.i2 = mask(i2);
    f.lew = mask(make_float2(hl * ((gyA == 0 || gyA == H - 1) ? 1.f : 2.f), hl * ((gyB == 0 || gyB == H - 1) ? 1.f : 2.f)));
    const float ln = hl * ((gx == 0 || gx == W - 1) ? 1.f : 2.f);
    f.lns = mask(make_float2(ln, ln));
    return f;
}

// One relaxed block update of a node pair:
//   x = D^{-1} (b - sum_K h_K (h_K . (z_j + z_k)) + sum_e w_e z_e),
//   z <- z + omega (x - z),
// the six elements as in node_sweep (E1 t0(x,y), E2 t1(x,y), E3 t0(x-1,y-1),
// E4 t1(x-1,y-1), E5 t0(x-1,y), E6 t1(x,y-1)), their paired records in e[];
// the values Z are indexed by the cell (row k = paired row k - 1).  The sums
// run in two independent chains (elements 1, 3, 5 and the E, W legs;
// elements 2, 4, 6 and the N, S legs) that are added at the end.
__device__ __forceinline__ void pair_update(const RecH2 (&e)[6], __half2* __restrict__ Z, int zp, int RW, int HPRW,
                                            __half2 om, PairState& n) {
    if (n.c < 0) return;
    const int c = n.c;
    const __half2* z0 = Z;
    const __half2* z1 = Z + zp;
    const __half2* z2 = Z + 2 * zp;
    const int iE = c + 1, iW = c - 1, iN = c + RW, iS = c - RW, iNE = c + RW + 1, iSW = c - RW - 1;
    const __half2 zE0 = z0[iE], zE1 = z1[iE], zE2 = z2[iE];
    const __half2 zW0 = z0[iW], zW1 = z1[iW], zW2 = z2[iW];
    const __half2 zN0 = z0[iN], zN1 = z1[iN], zN2 = z2[iN];
    const __half2 zS0 = z0[iS], zS1 = z1[iS], zS2 = z2[iS];
    const __half2 zNE0 = z0[iNE], zNE1 = z1[iNE], zNE2 = z2[iNE];
    const __half2 zSW0 = z0[iSW], zSW1 = z1[iSW], zSW2 = z2[iSW];
    // -h . (z_j + z_k) of each element
    auto dotn = [](const RecH2& r, __half2 a0, __half2 a1, __half2 a2, __half2 c0, __half2 c1, __half2 c2) {
        const __half2 s = __hfma2(r.h2, __hadd2(a2, c2), __hfma2(r.h1, __hadd2(a1, c1), __hmul2(r.h0, __hadd2(a0, c0))));
        return __hneg2(s);
    };
    const __half2 s1 = dotn(e[0], zE0, zE1, zE2, zNE0, zNE1, zNE2);
    const __half2 s2 = dotn(e[1], zN0, zN1, zN2, zNE0, zNE1, zNE2);
    const __half2 s3 = dotn(e[2], zSW0, zSW1, zSW2, zS0, zS1, zS2);
    const __half2 s4 = dotn(e[3], zSW0, zSW1, zSW2, zW0, zW1, zW2);
    const __half2 s5 = dotn(e[4], zW0, zW1, zW2, zN0, zN1, zN2);
    const __half2 s6 = dotn(e[5], zS0, zS1, zS2, zE0, zE1, zE2);
    // alpha edge weights: n-E = w of t0(x,y), n-N = w of t1(x,y), n-W = w of
    // t0(x-1,y), n-S = w of t1(x,y-1)
    __half2 a0 = __hfma2(s5, e[4].h0, __hfma2(s3, e[2].h0, __hfma2(s1, e[0].h0, n.b0)));
    __half2 a1 = __hfma2(s5, e[4].h1, __hfma2(s3, e[2].h1, __hfma2(s1, e[0].h1, n.b1)));
    __half2 a2 = __hfma2(s5, e[4].h2, __hfma2(s3, e[2].h2, __hfma2(s1, e[0].h2, n.b2)));
    __half2 c0 = __hfma2(s6, e[5].h0, __hfma2(s4, e[3].h0, __hmul2(s2, e[1].h0)));
    __half2 c1 = __hfma2(s6, e[5].h1, __hfma2(s4, e[3].h1, __hmul2(s2, e[1].h1)));
    __half2 c2 = __hfma2(s6, e[5].h2, __hfma2(s4, e[3].h2, __hmul2(s2, e[1].h2)));
    a0 = __hfma2(e[0].w, zE0, __hfma2(e[4].w, zW0, a0));
    a1 = __hfma2(e[0].w, zE1, __hfma2(e[4].w, zW1, a1));
    a2 = __hfma2(n.lew, __hadd2(zE2, zW2), a2);
    c0 = __hfma2(e[1].w, zN0, __hfma2(e[5].w, zS0, c0));
    c1 = __hfma2(e[1].w, zN1, __hfma2(e[5].w, zS1, c1));
    c2 = __hfma2(n.lns, __hadd2(zN2, zS2), c2);
    __half2 x0, x1, x2;
    block_solve_h2(n.B, __hadd2(a0, c0), __hadd2(a1, c1), __hadd2(a2, c2), x0, x1, x2);
    n.z0 = __hfma2(om, __hsub2(x0, n.z0), n.z0);
    n.z1 = __hfma2(om, __hsub2(x1, n.z1), n.z1);
    n.z2 = __hfma2(om, __hsub2(x2, n.z2), n.z2);
    Z[c] = n.z0;
    Z[c + zp] = n.z1;
    Z[c + 2 * zp] = n.z2;
    if (n.seam) {
        // the seam ghost (the other lane of the ghost word is the zero ring)
        const __half zero = __float2half(0.f);
        const int g = n.seam == 1 ? c - HPRW : c + HPRW;
        auto gh = [&](__half2 v) {
            return n.seam == 1 ? __halves2half2(zero, __low2half(v)) : __halves2half2(__high2half(v), zero);
        };
        Z[g] = gh(n.z0);
        Z[g + zp] = gh(n.z1);
        Z[g + 2 * zp] = gh(n.z2);
    }
}

// The six paired records (E1..E6) of the node pair at cell c.
__device__ __forceinline__ void pair_records(const RecH2* __restrict__ P0, const RecH2* __restrict__ P1, int c,
                                             int RW, RecH2 (&e)[6]) {
    e[0] = P0[c];
    e[1] = P1[c];
    e[2] = P0[c - RW - 1];
    e[3] = P1[c - RW - 1];
    e[4] = P0[c - 1];
    e[5] = P1[c - RW];
}

// Writes the paired values of a node pair (and their seam ghosts).
__device__ __forceinline__ void pair_store(__half2* __restrict__ Z, int zp, int HPRW, int c, int seam, __half2 v0,
                                           __half2 v1, __half2 v2) {
    Z[c] = v0;
    Z[c + zp] = v1;
    Z[c + 2 * zp] = v2;
    if (seam) {
        const __half zero = __float2half(0.f);
        const int g = seam == 1 ? c - HPRW : c + HPRW;
        auto gh = [&](__half2 v) {
            return seam == 1 ? __halves2half2(zero, __low2half(v)) : __halves2half2(__high2half(v), zero);
        };
        Z[g] = gh(v0);
        Z[g + zp] = gh(v1);
        Z[g + 2 * zp] = gh(v2);
    }
}

template <int TXC, int TYC, int OVC>
__global__ void __launch_bounds__(384, 1) k_schwarz_h2(const SchwarzParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ DF sh_red[64];
    __shared__ float sh_max[16];
    __shared__ float sh_part[32];  // per-warp r.r (0..15) and r.z (16..31) of the pending item
    __shared__ int sh_last, sh_fail, sh_more;
    __shared__ float sh_a;
    const int NT = blockDim.x;
    const int Tx = TXC ? TXC : P.Tx, Ty = TXC ? TYC : P.Ty, ov = TXC ? OVC : P.ov;
    const int RW = sch_rw(Tx, ov), HP = h2_hp(Ty, ov), cpad = sch_cpad(ov);
    const int nz = RW * (HP + 2), nr = RW * (HP + 1), HPRW = HP * RW;
    const int nstage = P.nstage;
    const H2Layout L = h2_layout(Tx, Ty, ov, nstage);
    unsigned char* base = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bar);
    __half2* Zs = reinterpret_cast<__half2*>(base + L.zs);
    const unsigned box_rq = (unsigned)(3 * (size_t)Tx * Ty * sizeof(float));
    const unsigned box_p = (unsigned)(nr * sizeof(RecH2));

    if (threadIdx.x == 0) {
        sh_fail = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    // the ring (and the other lane of each ghost word) is never written: the
    // Dirichlet zeros of every item
    for (int i = threadIdx.x; i < 3 * nz; i += NT) Zs[i] = __float2half2_rn(0.f);
    __syncthreads();

    auto issue = [&](const int4 ti, int s) {
        const CUtensorMap* tm = P.tmaps + (size_t)ti.x * TM_PER_PAIR;
        const int x0 = ti.y * Tx, y0 = ti.z * Ty;
        const bool need_q = !P.first && !P.apply_only;
        unsigned char* st = base + L.stage0 + (size_t)s * L.stage_bytes;
        bulk_wait_read();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bars[s], 2 * box_p + box_rq + (need_q ? box_rq : 0u) + (unsigned)P.tx_extra);
        // records as pairs of 8-byte units; row k of the plane is image row k - ov - 1
        const int cx = (x0 - cpad) * 2, cy = y0;
        tma_load_2d(st + L.p0, tm + TM_P0, cx, cy, &bars[s]);
        tma_load_2d(st + L.p1, tm + TM_P1, cx, cy, &bars[s]);
        tma_load_3d(st + L.rs, tm + TM_R, x0, y0, 0, &bars[s]);
        if (need_q) tma_load_3d(st + L.qs, tm + TM_Q, x0, y0, 0, &bars[s]);
    };
    const int G = gridDim.x;
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
    auto advance = [&](int t, int4& ti) {
        while (t < P.ntiles) {
            ti = P.tiles[t];
            if (!pair_done(ti.x)) return t;
            t += G;
        }
        return t;
    };
    uint32_t tab[3];
#pragma unroll
    for (int col = 0; col < 3; ++col) tab[col] = P.ntab[col * NT + threadIdx.x];
    const float hl = 0.5f * (float)P.lam;
    const float om = (float)P.omega;
    const __half2 om2 = __float2half2_rn(om);

    // the pair's size and the step a of a work item, read one item ahead
    struct ItemScalars {
        int W, H;
        float a;
    };
    // one pair: the step a = r.z / p.q from the apply's fixed-point p.q
    // (pq_fix_shift), formed by thread 0 of every CTA (all take the same a);
    // the last CTA stores p.q and a and clears the sum
    const bool pq_here = P.pq_fixed && !P.first && !P.apply_only && P.npairs == 1;
    double pq_val = 0.0, a_val = 0.0;  // thread 0
    int pq_bad = 0;
    auto item_scalars = [&](const int4 w) {
        ItemScalars r;
        r.W = P.pairs[w.x].W;
        r.H = P.pairs[w.x].H;
        // one FP64 conversion per warp (the FP64 pipe is narrow), broadcast
        float a = 0.f;
        if ((threadIdx.x & 31) == 0 && !P.first && !P.apply_only && !pq_here) a = (float)P.sc[w.x].a;
        r.a = pq_here ? sh_a : __shfl_sync(0xffffffffu, a, 0);
        return r;
    };
    // the store of an item's z (and updated r) and its partial sums run after
    // the first barrier of the next item (with two stages), when every
    // thread's writes to them are complete
    struct Pending {
        int pair, x0, y0, w, stage;
        bool need_q;
    };
    Pending pend;
    pend.pair = -1;
    // Unless a coarse level reads the items' partials: one partial per pair
    // and CTA, the sum over the CTA's items of the pair (in their order, in
    // double-float), in the slot of the CTA's first item of the pair.  The
    // CTA with index c takes the items c, c + G, c + 2G, ... (done pairs
    // skipped), so a pair's slots are its first min(items, G) item indices
    // and the last CTA sums at most G values per pair.
    const bool per_cta = !P.defer;
    DF cta_rr{0.f, 0.f}, cta_rz{0.f, 0.f};
    int cta_pair = -1, cta_slot = 0;
    auto cta_write = [&]() {
        P.partial[2 * (long long)cta_slot] = df_to_double(cta_rr);
        P.partial[2 * (long long)cta_slot + 1] = df_to_double(cta_rz);
    };
    auto flush = [&](const Pending& q) {
        unsigned char* sq = base + L.stage0 + (size_t)q.stage * L.stage_bytes;
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const CUtensorMap* tm = P.tmaps + (size_t)q.pair * TM_PER_PAIR;
            tma_store_3d(tm + TM_Z, q.x0, q.y0, 0, sq + L.qs);
            if (q.need_q) tma_store_3d(tm + TM_R, q.x0, q.y0, 0, sq + L.rs);
            bulk_commit();
        }
        // the item's r.r and r.z from the per-warp sums in fixed order, in
        // FP32 (the FP64 pipe is narrow) (warp 1: thread 0 issues the
        // stores); they are summed per pair over the CTA's items (in
        // double-float, in the items' order) and written when the CTA moves
        // on to another pair and at its end
        if (!P.apply_only && (threadIdx.x >> 5) == 1) {
            const int l = threadIdx.x & 31;
            const bool w = l < (NT >> 5);
            const float a2 = warp_sum(w ? sh_part[l] : 0.f), b2 = warp_sum(w ? sh_part[16 + l] : 0.f);
            if (l == 0) {
                if (per_cta) {
                    if (q.pair != cta_pair) {
                        if (cta_pair >= 0) cta_write();
                        cta_pair = q.pair;
                        cta_slot = q.w;
                        cta_rr = DF{a2, 0.f};
                        cta_rz = DF{b2, 0.f};
                    } else {
                        cta_rr = cta_rr + DF{a2, 0.f};
                        cta_rz = cta_rz + DF{b2, 0.f};
                    }
                } else {
                    P.partial[2 * (long long)q.w] = (double)a2;
                    P.partial[2 * (long long)q.w + 1] = (double)b2;
                }
            }
        }
    };

    int4 ti = make_int4(0, 0, 0, 0), tin = make_int4(0, 0, 0, 0);
    int t = advance(blockIdx.x, ti);
    int tn = (t < P.ntiles) ? advance(t + G, tin) : P.ntiles;
    if (t < P.ntiles && threadIdx.x == 0) issue(ti, 0);
    if (pq_here) {  // while the first item's copies are in flight
        if (threadIdx.x == 0) {
            const PairScalars* s0 = P.sc;
            const double rz = s0->rz;
            const long long fix = s0->pq_fix;
            pq_bad = s0->pad[1];
            pq_val = (double)fix * __longlong_as_double((long long)(1023 - pq_fix_shift(rz)) << 52);
            a_val = (!pq_bad && pq_val > 0.0 && isfinite(rz)) ? rz / pq_val : 0.0;
            sh_a = (float)a_val;
        }
        __syncthreads();
    }
    ItemScalars cur = {0, 0, 0.f}, nxt = {0, 0, 0.f};
    if (t < P.ntiles) cur = item_scalars(ti);
    unsigned phase[2] = {0u, 0u};
    int s = 0;
    for (; t < P.ntiles;) {
        const int tc = tn + G;
        int4 tic = make_int4(0, 0, 0, 0);
        if (tn < P.ntiles && tc < P.ntiles) tic = P.tiles[tc];
        if (tn < P.ntiles) nxt = item_scalars(tin);
        if (threadIdx.x == 0 && !mbar_wait_phase_bounded(&bars[s], phase[s], P.spin_limit)) {
            sh_fail = 1;
            atomicOr(P.err, 1);
        }
        __syncthreads();
        if (sh_fail) {
            if (threadIdx.x == 0) mbar_wait_phase_bounded(&bars[s], phase[s], P.spin_limit);
            break;
        }
        if (!mbar_wait_phase_bounded(&bars[s], phase[s], P.spin_limit)) atomicOr(P.err, 1);
        phase[s] ^= 1u;
        if (pend.pair >= 0) {
            flush(pend);
            pend.pair = -1;
        }
        unsigned char* st = base + L.stage0 + (size_t)s * L.stage_bytes;
        const RecH2* P0s = reinterpret_cast<const RecH2*>(st + L.p0);
        const RecH2* P1s = reinterpret_cast<const RecH2*>(st + L.p1);
        float* Rs = reinterpret_cast<float*>(st + L.rs);
        const float* Qs = reinterpret_cast<const float*>(st + L.qs);
        const int pair = ti.x;
        const int W = cur.W, H = cur.H;
        const int x0 = ti.y * Tx, y0 = ti.z * Ty;
        const int tw = min(Tx, W - x0), th = min(Ty, H - y0);
        const int ex0 = max(x0 - ov, 0), ex1 = min(x0 + tw + ov, W);
        const int ey0 = max(y0 - ov, 0), ey1 = min(y0 + th + ov, H);
        const bool need_q = !P.first && !P.apply_only;
        const float a = cur.a;
        const int plane = Tx * Ty;
        // ---- setup in FP32, both lanes of a pair at once in packed (float2)
        // arithmetic: diagonal blocks and their LDL^T factors, right-hand sides
        // (r <- r - a q on the owned nodes), the first Jacobi step and its
        // largest entry
        float rr = 0.f, zmax = 0.f;
        PairState ns[3];
        RecH2 rec1[6];
        float2 bf[3][3];
        float2 xj[3];
        const float2 zero2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int col = 0; col < 3; ++col) {
            PairState& n = ns[col];
            const uint32_t e = tab[col];
            n.c = -1;
            n.seam = 0;
            const __half2 hz = __float2half2_rn(0.f);
            n.B.i0 = n.B.l10 = n.B.l20 = n.B.i1 = n.B.l21 = n.B.i2 = n.lew = n.lns = hz;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                bf[col][k] = zero2;
                if (col == 0) xj[k] = zero2;
            }
            if (e == 0xffffffffu) continue;
            const int li = (int)(e & 0xffffu), lj = (int)(e >> 16);
            const int c = (lj + 1) * RW + (li + cpad - ov);
            // the pair's z accesses lie in [c - RW - 1, c + RW + 1] of each plane,
            // its ghost at c -+ HP RW, its records in [c - RW - 1, c]
            if (!OF_CHECK(P.err, c - RW - 1, nr) || !OF_CHECK(P.err, c, nr) || !OF_CHECK(P.err, c + RW + 1, nz) ||
                (lj == HP - 1 && !OF_CHECK(P.err, c - HPRW, nz)) || (lj == 0 && !OF_CHECK(P.err, c + HPRW, nz)))
                continue;
            n.c = c;
            n.seam = (lj == HP - 1) ? 1 : (lj == 0 ? 2 : 0);
            RecH2 rec[6];
            pair_records(P0s, P1s, c, RW, rec);
            if (col == 1) {
#pragma unroll
                for (int k = 0; k < 6; ++k) rec1[k] = rec[k];  // colour 1 (half the visits) keeps its records
            }
            const int gx = x0 - ov + li, gyA = y0 - ov + lj, gyB = gyA + HP;
            const bool inx = gx >= ex0 && gx < ex1;
            const bool vA = inx && gyA >= ey0 && gyA < ey1, vB = inx && gyB >= ey0 && gyB < ey1;
            if (!vA && !vB) continue;  // clipped: factors and values stay zero
            const FacF2 f = pair_factors(rec, gx, gyA, gyB, vA, vB, W, H, hl);
            n.B.i0 = __float22half2_rn(f.i0);
            n.B.l10 = __float22half2_rn(f.l10);
            n.B.l20 = __float22half2_rn(f.l20);
            n.B.i1 = __float22half2_rn(f.i1);
            n.B.l21 = __float22half2_rn(f.l21);
            n.B.i2 = __float22half2_rn(f.i2);
            n.lew = __float22half2_rn(f.lew);
            n.lns = __float22half2_rn(f.lns);
            // right-hand sides on the owned nodes (r <- r - a q)
            float bv[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
            bool any = false;
#pragma unroll
            for (int Ln = 0; Ln < 2; ++Ln) {
                const int gy = Ln ? gyB : gyA;
                if (!(gx >= x0 && gx < x0 + tw && gy >= y0 && gy < y0 + th)) continue;
                if (!OF_CHECK(P.err, (gy - y0) * Tx + (gx - x0), plane)) continue;
                const int si = (gy - y0) * Tx + (gx - x0);
                float v0 = Rs[si], v1 = Rs[si + plane], v2 = Rs[si + 2 * plane];
                if (need_q) {
                    v0 -= a * Qs[si];
                    v1 -= a * Qs[si + plane];
                    v2 -= a * Qs[si + 2 * plane];
                    Rs[si] = v0;
                    Rs[si + plane] = v1;
                    Rs[si + 2 * plane] = v2;
                }
                bv[Ln][0] = v0;
                bv[Ln][1] = v1;
                bv[Ln][2] = v2;
                rr += v0 * v0 + v1 * v1 + v2 * v2;
                any = true;
            }
            if (!any) continue;
#pragma unroll
            for (int k = 0; k < 3; ++k) bf[col][k] = make_float2(bv[0][k], bv[1][k]);
            // the first Jacobi step z = D^{-1} b, both lanes
            auto neg = [](float2 v) { return make_float2(-v.x, -v.y); };
            const float2 b0 = bf[col][0], b1 = bf[col][1], b2 = bf[col][2];
            const float2 y1 = __ffma2_rn(neg(f.l10), b0, b1);
            const float2 y2 = __ffma2_rn(neg(f.l21), y1, __ffma2_rn(neg(f.l20), b0, b2));
            const float2 q2 = __fmul2_rn(y2, f.i2);
            const float2 q1 = __ffma2_rn(neg(f.l21), q2, __fmul2_rn(y1, f.i1));
            const float2 q0 = __ffma2_rn(neg(f.l20), q2, __ffma2_rn(neg(f.l10), q1, __fmul2_rn(b0, f.i0)));
            zmax = fmaxf(zmax, fmaxf(fmaxf(fabsf(q0.x), fabsf(q0.y)),
                                     fmaxf(fmaxf(fabsf(q1.x), fabsf(q1.y)), fmaxf(fabsf(q2.x), fabsf(q2.y)))));
            if (col == 0) {
                xj[0] = q0;
                xj[1] = q1;
                xj[2] = q2;
            }
        }
        // the tile's scale: the largest entry of the first Jacobi step
        {
            const float wm = warp_max(zmax);
            if ((threadIdx.x & 31) == 0) sh_max[threadIdx.x >> 5] = wm;
        }
        __syncthreads();
        float m = 0.f;
        for (int w = 0; w < (NT >> 5); ++w) m = fmaxf(m, sh_max[w]);
        const bool mok = m > 0.f && m <= 3.0e38f;  // false for 0, inf and NaN
        const float scl = mok ? 1.f / m : 1.f, unscl = mok ? m : 1.f;
        const float omj = P.sweeps > 0 ? om : 1.f;
#pragma unroll
        for (int col = 0; col < 3; ++col) {
            PairState& n = ns[col];
            const float2 sc2 = make_float2(scl, scl), oj2 = make_float2(omj * scl, omj * scl);
            n.b0 = __float22half2_rn(__fmul2_rn(bf[col][0], sc2));
            n.b1 = __float22half2_rn(__fmul2_rn(bf[col][1], sc2));
            n.b2 = __float22half2_rn(__fmul2_rn(bf[col][2], sc2));
            if (col == 0) {
                // the first colour step from z = 0: (relaxed) block Jacobi
                n.z0 = __float22half2_rn(__fmul2_rn(xj[0], oj2));
                n.z1 = __float22half2_rn(__fmul2_rn(xj[1], oj2));
                n.z2 = __float22half2_rn(__fmul2_rn(xj[2], oj2));
            } else {
                n.z0 = n.z1 = n.z2 = __float2half2_rn(0.f);
            }
            if (n.c >= 0) pair_store(Zs, nz, HPRW, n.c, n.seam, n.z0, n.z1, n.z2);
        }
        __syncthreads();
        if (nstage == 2 && tn < P.ntiles && threadIdx.x == 0) issue(tin, s ^ 1);

        // ---- sweeps (colour order 0,1,2,1,0,...,0; the first 0 was the Jacobi
        // step above); the last visit of each colour writes the owned z,
        // scaled back, into this stage's q buffer and accumulates r.z in FP32
        float rz = 0.f;
        float* zo = reinterpret_cast<float*>(st + L.qs);
        auto emit = [&](const PairState& n) {
            if (n.c < 0) return;
            const int row = n.c / RW;
            const int li = n.c - row * RW - cpad + ov, lj = row - 1;
#pragma unroll
            for (int Ln = 0; Ln < 2; ++Ln) {
                const int ox = li - ov, oy = lj + Ln * HP - ov;
                if (ox < 0 || ox >= tw || oy < 0 || oy >= th || !OF_CHECK(P.err, oy * Tx + ox, plane)) continue;
                const int si = oy * Tx + ox;
                const float v0 = h_lane(n.z0, Ln) * unscl, v1 = h_lane(n.z1, Ln) * unscl,
                            v2 = h_lane(n.z2, Ln) * unscl;
                zo[si] = v0;
                zo[si + plane] = v1;
                zo[si + 2 * plane] = v2;
                rz += Rs[si] * v0 + Rs[si + plane] * v1 + Rs[si + 2 * plane] * v2;
            }
        };
// colour 1 (half of all visits) keeps its records in registers (set up above)
#define OF_H2STEP(col, last, sync)                                            \
    {                                                                         \
        if (col == 1) {                                                       \
            pair_update(rec1, Zs, nz, RW, HPRW, om2, ns[1]);                  \
        } else if (ns[col].c >= 0) {                                          \
            RecH2 e_[6];                                                      \
            pair_records(P0s, P1s, ns[col].c, RW, e_);                        \
            pair_update(e_, Zs, nz, RW, HPRW, om2, ns[col]);                  \
        }                                                                     \
        if (last) emit(ns[col]);                                              \
        if (sync) __syncthreads();                                            \
    }
        OF_H2STEP(1, false, true)
        OF_H2STEP(2, P.sweeps == 1, true)
        OF_H2STEP(1, P.sweeps == 1, true)
        for (int sw = 1; sw < P.sweeps; ++sw) {
            const bool lastsw = (sw == P.sweeps - 1);
            OF_H2STEP(0, false, true)
            OF_H2STEP(1, false, true)
            OF_H2STEP(2, lastsw, true)
            OF_H2STEP(1, lastsw, true)
        }
        // the last step's barrier is the next item's first one (or the one
        // before the flush below)
        OF_H2STEP(0, true, false)
#undef OF_H2STEP

        const float wrr = warp_sum(rr), wrz = warp_sum(rz);
        if ((threadIdx.x & 31) == 0) {
            sh_part[threadIdx.x >> 5] = wrr;
            sh_part[16 + (threadIdx.x >> 5)] = wrz;
        }
        pend.pair = pair;
        pend.x0 = x0;
        pend.y0 = y0;
        pend.w = ti.w;
        pend.stage = s;
        pend.need_q = need_q;
        if (nstage == 1) {
            // one stage: the store must leave it before the next item's loads
            __syncthreads();
            flush(pend);
            pend.pair = -1;
        }
        t = tn;
        ti = tin;
        tn = tc;
        cur = nxt;
        tin = tic;
        if (tn < P.ntiles && pair_done(tin.x)) tn = advance(tn + G, tin);
        if (nstage == 2) s ^= 1;
        else if (t < P.ntiles && threadIdx.x == 0) issue(ti, 0);
    }
    if (pend.pair >= 0) {
        __syncthreads();
        flush(pend);
    }
    if (per_cta && !P.apply_only && threadIdx.x == 32 && cta_pair >= 0) cta_write();
    if (threadIdx.x == 0) bulk_wait_all();
    if (P.apply_only || P.defer) return;
    if (!arrive_last(P.counter, gridDim.x, &sh_last)) return;
    // the last CTA: r.r and r.z of each pair from its items' partials (fixed
    // order, double-float), the pair's CG scalars, the loop condition.  The
    // scalars and the error word are read before the partials so that their
    // loads overlap; no other CTA of this launch writes them any more.
    const int err_now = (threadIdx.x == 0) ? *(volatile int*)P.err : 0;
    if (P.npairs == 1) {
        PairScalars s0;
        if (threadIdx.x == 0) s0 = P.sc[0];
        double t_rr = 0.0, t_rz = 0.0;
        df_ordered_sum2<4>(P.partial, min(P.ntiles, (int)gridDim.x), t_rr, t_rz, sh_red);  // the CTAs' partials
        if (threadIdx.x == 0) {
            if (!s0.done) {
                if (pq_here) {
                    // the step of this iteration (what the apply's own reduction stores otherwise)
                    s0.pq = pq_val;
                    s0.a = a_val;
                    if (pq_bad || !(pq_val > 0.0) || !isfinite(s0.rz)) {
                        s0.a = 0.0;
                        s0.done = 1;
                        s0.status = 6;
                    }
                }
                if (!s0.done) precond_finalize(&s0, t_rr, t_rz, P.first);
            }
            s0.pq_fix = 0;  // the next apply's sum starts from zero
            s0.pad[1] = 0;
            P.sc[0] = s0;
            sh_more = s0.done ? 0 : 1;  // another iteration
        }
    } else {
        // one warp per pair
        if (threadIdx.x == 0) sh_more = 0;
        __syncthreads();
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = NT >> 5;
        for (int pi = w; pi < P.npairs; pi += nw) {
            PairScalars* sp = P.sc + pi;
            if (sp->done) continue;
            const PairDesc pd = P.pairs[pi];
            const int ntp = min(pd.tiles_x * pd.tiles_y, (int)gridDim.x);  // the pair's CTA partials
            const double2* q = reinterpret_cast<const double2*>(P.partial) + pd.tile0;
            DF a0{0.f, 0.f}, a1{0.f, 0.f}, b0{0.f, 0.f}, b1{0.f, 0.f};
            int i = l;
            for (; i + 32 < ntp; i += 64) {
                const double2 u = __ldcg(q + i), v = __ldcg(q + i + 32);
                a0 = a0 + df_from_double(u.x);
                b0 = b0 + df_from_double(u.y);
                a1 = a1 + df_from_double(v.x);
                b1 = b1 + df_from_double(v.y);
            }
            if (i < ntp) {
                const double2 u = __ldcg(q + i);
                a0 = a0 + df_from_double(u.x);
                b0 = b0 + df_from_double(u.y);
            }
            const DF x = df_warp_sum(a0 + a1), y = df_warp_sum(b0 + b1);
            if (l == 0) {
                precond_finalize(sp, df_to_double(x), df_to_double(y), P.first);
                if (!sp->done) atomicOr(&sh_more, 1);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (P.use_cond) cudaGraphSetConditional(P.cond, (sh_more && !err_now) ? 1u : 0u);
        *P.counter = 0u;
    }
}

}  // namespace ofk
