// Overlapping Schwarz preconditioner (Section 3.2, Eq. schwarz), one CTA per
// subdomain, fused with the residual update of the Krylov loop.
//
// Subdomain i owns a tile T_x x T_y of nodes; its extended tile adds `o`
// node layers on every side that is not on the image boundary (the overlap
// Sigma_ij of Section 3.2).  The local problem is the global operator
// restricted to the extended tile with homogeneous Dirichlet values outside
// it (the algebraic form of the Dirichlet transmission condition on
// Gamma_ij) and the natural Neumann condition on the image boundary.  It is
// solved approximately by `s` symmetric 3-colour block Gauss-Seidel sweeps
// from zero (colours (x+y) mod 3 make the 7-point stencil conflict free;
// the colour order 0,1,2,1,0,1,2,1,0,... is a palindrome, so the sweep
// operator is symmetric).  For CG the preconditioner must be symmetric, so
// the subdomain right-hand side is the residual on the owned nodes only and
// only the owned part of the local solution is kept:
//   z = sum_i R~_i^T  A_i^{-1}(approx)  R~_i r        (R~_i: owned nodes)
// which is symmetric positive definite (block diagonal over owned tiles of
// SPD blocks).  With sweeps = 0 and overlap 0 it is node-block Jacobi.
//
// Staging: the coefficient window (frames over the extended tile plus a
// one-node halo, alpha of every square touching it) and the owned tiles of r
// and q arrive by TMA (cp.async.bulk.tensor) on one mbarrier with a bounded
// wait.  The update r <- r - a q, the norms r.r and r.z (FP64 partials,
// deterministic last-CTA reduction per pair) are fused in.
#pragma once
#include <cuda.h>
#include "of_common.cuh"

namespace ofk {

enum { TM_F1 = 0, TM_F2 = 1, TM_AL = 2, TM_R = 3, TM_Q = 4, TM_PER_PAIR = 5 };

struct SchwarzParams {
    const PairDesc* pairs;
    const int4* tiles;        // per work item: (pair, tile x, tile y, global tile index)
    const CUtensorMap* tmaps; // [batch][TM_PER_PAIR], 64-byte aligned
    PairScalars* sc;
    double* partial;          // [ntiles][2]
    unsigned* counter;        // [batch]
    int* err;                 // device error word (bit 0: TMA wait timed out)
    void* r;                  // inner residual planes (written back on owned nodes)
    void* z;                  // preconditioned residual planes (owned nodes)
    double lam;
    int Tx, Ty, ov, sweeps;
    int first;                // no r update (start of a pass): z = M r only
    int apply_only;           // of_precondition: z = M r, no scalars
    long long spin_limit;     // bounded mbarrier wait, in clock64 cycles
};

__host__ __device__ inline int sch_padl(int ov) { return ((ov + 1) + 3) & ~3; }
__host__ __device__ inline int sch_bw(int Tx, int ov) { return (sch_padl(ov) + Tx + ov + 1 + 3) & ~3; }
__host__ __device__ inline int sch_bh(int Ty, int ov) { return Ty + 2 * ov + 2; }

template <typename R>
__host__ __device__ inline size_t sch_smem_bytes(int Tx, int Ty, int ov) {
    const int BW = sch_bw(Tx, ov), BH = sch_bh(Ty, ov);
    const size_t zw = (size_t)(Tx + 2 * ov + 2), zh = (size_t)(Ty + 2 * ov + 2);
    auto al = [](size_t b) { return (b + 127) & ~(size_t)127; };
    size_t s = 256;                                   // alignment slack + mbarrier
    s += al(3 * (size_t)Tx * Ty * sizeof(R));         // R
    s += al(3 * (size_t)Tx * Ty * sizeof(R));         // Q
    s += al(3 * zw * zh * sizeof(R));                 // Z (zero ring)
    s += 2 * al((size_t)BW * BH * sizeof(R));         // F1, F2
    s += al(2 * (size_t)BW * BH * sizeof(R));         // AL
    return s;
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

// Bounded wait on phase 0 of the staging barrier: returns false after
// `limit` cycles (the caller records the timeout and stops).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, 0)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

template <typename R> __device__ __forceinline__ R rcp(R x) { return R(1) / x; }

// One block Gauss-Seidel update of node (gx, gy): solve the node's 3x3 block
// of the local operator for the new z, with the neighbours' current z.
template <typename R>
__device__ __forceinline__ void node_update(int gx, int gy, int W, int H, const R* F1, const R* F2, const R* AL,
                                            int ci, int BW, R* Z, int zi, int ZW, int zplane, R r0, R r1, R r2,
                                            R lam) {
    const R third = R(1) / R(3), w24 = R(1) / R(24), w12 = R(1) / R(12), h = R(OF_STIFF_HALF);
    // frames at n, E, W, N, S, NE, SW
    const R f2n = F2[ci], f2E = F2[ci + 1], f2W = F2[ci - 1], f2N = F2[ci + BW], f2S = F2[ci - BW];
    const R f2NE = F2[ci + BW + 1], f2SW = F2[ci - BW - 1];
    const R f1n = F1[ci], f1E = F1[ci + 1], f1W = F1[ci - 1], f1N = F1[ci + BW], f1S = F1[ci - BW];
    const R f1NE = F1[ci + BW + 1], f1SW = F1[ci - BW - 1];
    // squares (x,y), (x-1,y-1), (x-1,y), (x,y-1)
    const bool vc = (gx < W - 1) && (gy < H - 1);
    const bool vsw = (gx >= 1) && (gy >= 1);
    const bool vw = (gx >= 1) && (gy < H - 1);
    const bool vs = (gx < W - 1) && (gy >= 1);
    const R a1 = vc ? AL[2 * ci] : R(0), a2 = vc ? AL[2 * ci + 1] : R(0);
    const R a3 = vsw ? AL[2 * (ci - BW - 1)] : R(0), a4 = vsw ? AL[2 * (ci - BW - 1) + 1] : R(0);
    const R a5 = vw ? AL[2 * (ci - 1)] : R(0);
    const R a6 = vs ? AL[2 * (ci - BW) + 1] : R(0);
    // neighbours' z
    const R* z0 = Z;
    const R* z1 = Z + zplane;
    const R* z2 = Z + 2 * zplane;
    const int iE = zi + 1, iW = zi - 1, iN = zi + ZW, iS = zi - ZW, iNE = zi + ZW + 1, iSW = zi - ZW - 1;
    const R zE0 = z0[iE], zE1 = z1[iE], zE2 = z2[iE];
    const R zW0 = z0[iW], zW1 = z1[iW], zW2 = z2[iW];
    const R zN0 = z0[iN], zN1 = z1[iN], zN2 = z2[iN];
    const R zS0 = z0[iS], zS1 = z1[iS], zS2 = z2[iS];
    const R zNE0 = z0[iNE], zNE1 = z1[iNE], zNE2 = z2[iNE];
    const R zSW0 = z0[iSW], zSW1 = z1[iSW], zSW2 = z2[iSW];

    R b0 = r0, b1 = r1, b2 = r2;
    R D00 = 0, D01 = 0, D02 = 0, D11 = 0, D12 = 0, D22 = 0;
    auto elem = [&](bool v, R gx_, R gy_, R gm_, R s0, R s1, R s2) {
        if (!v) return;
        const R s = gx_ * s0 + gy_ * s1 + gm_ * s2;
        const R k = s * w24;
        b0 -= k * gx_; b1 -= k * gy_; b2 -= k * gm_;
        D00 += w12 * gx_ * gx_; D01 += w12 * gx_ * gy_; D02 += w12 * gx_ * gm_;
        D11 += w12 * gy_ * gy_; D12 += w12 * gy_ * gm_; D22 += w12 * gm_ * gm_;
    };
    // E1: square (x,y) t=0, others E, NE
    elem(vc, f2E - f2n, f2NE - f2E, -(f1n + f1E + f1NE) * third, zE0 + zNE0, zE1 + zNE1, zE2 + zNE2);
    // E2: square (x,y) t=1, others N, NE
    elem(vc, f2NE - f2N, f2N - f2n, -(f1n + f1N + f1NE) * third, zN0 + zNE0, zN1 + zNE1, zN2 + zNE2);
    // E3: square (x-1,y-1) t=0, others SW, S
    elem(vsw, f2S - f2SW, f2n - f2S, -(f1SW + f1S + f1n) * third, zSW0 + zS0, zSW1 + zS1, zSW2 + zS2);
    // E4: square (x-1,y-1) t=1, others SW, W
    elem(vsw, f2n - f2W, f2W - f2SW, -(f1SW + f1W + f1n) * third, zSW0 + zW0, zSW1 + zW1, zSW2 + zW2);
    // E5: square (x-1,y) t=0, others W, N
    elem(vw, f2n - f2W, f2N - f2n, -(f1W + f1n + f1N) * third, zW0 + zN0, zW1 + zN1, zW2 + zN2);
    // E6: square (x,y-1) t=1, others S, E
    elem(vs, f2E - f2n, f2n - f2S, -(f1S + f1n + f1E) * third, zS0 + zE0, zS1 + zE1, zS2 + zE2);
    // stiffness legs: n-E (E1, E6), n-N (E2, E5), n-W (E4, E5), n-S (E3, E6)
    const R wE = h * (a1 + a6), wN = h * (a2 + a5), wWe = h * (a4 + a5), wS = h * (a3 + a6);
    const R lE = h * lam * (R(vc) + R(vs)), lN = h * lam * (R(vc) + R(vw));
    const R lW = h * lam * (R(vsw) + R(vw)), lS = h * lam * (R(vsw) + R(vs));
    b0 += wE * zE0 + wN * zN0 + wWe * zW0 + wS * zS0;
    b1 += wE * zE1 + wN * zN1 + wWe * zW1 + wS * zS1;
    b2 += lE * zE2 + lN * zN2 + lW * zW2 + lS * zS2;
    D00 += wE + wN + wWe + wS;
    D11 += wE + wN + wWe + wS;
    D22 += lE + lN + lW + lS;
    // 3x3 SPD solve by LDL^T
    const R i0 = rcp(D00);
    const R l10 = D01 * i0, l20 = D02 * i0;
    const R d1 = D11 - l10 * D01;
    const R i1 = rcp(d1);
    const R l21 = (D12 - l20 * D01) * i1;
    const R d2 = D22 - l20 * D02 - l21 * l21 * d1;
    const R i2 = rcp(d2);
    const R y0 = b0, y1 = b1 - l10 * y0, y2 = b2 - l20 * y0 - l21 * y1;
    const R x2 = y2 * i2;
    const R x1 = y1 * i1 - l21 * x2;
    const R x0 = y0 * i0 - l10 * x1 - l20 * x2;
    Z[zi] = x0;
    Z[zi + zplane] = x1;
    Z[zi + 2 * zplane] = x2;
}

template <typename R, int NT>
__global__ void __launch_bounds__(NT) k_schwarz(const SchwarzParams P) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ double sh_red[NT / 32];
    __shared__ int sh_last, sh_fail;
    const int4 ti = P.tiles[blockIdx.x];
    const int pair = ti.x;
    if (!P.apply_only && P.sc[pair].done) return;  // uniform over the pair's tiles
    const PairDesc pd = P.pairs[pair];
    const int W = pd.W, H = pd.H, pitch = pd.pitch;
    const long long plane = (long long)H * pitch;
    const int Tx = P.Tx, Ty = P.Ty, ov = P.ov;
    const int x0 = ti.y * Tx, y0 = ti.z * Ty;
    const int tw = min(Tx, W - x0), th = min(Ty, H - y0);
    const int BW = sch_bw(Tx, ov), BH = sch_bh(Ty, ov);
    const int xs = x0 - sch_padl(ov), ys = y0 - ov - 1;
    const int ZW = Tx + 2 * ov + 2, ZH = Ty + 2 * ov + 2;
    const int zplane = ZW * ZH;
    const bool need_q = !P.first && !P.apply_only;

    auto al = [](size_t b) { return (b + 127) & ~(size_t)127; };
    // TMA destinations on 128-byte boundaries whatever the base alignment
    unsigned char* base = smem + ((128u - (smem_u32(smem) & 127u)) & 127u);
    uint64_t* bar = reinterpret_cast<uint64_t*>(base);
    size_t off = 128;
    R* Rs = reinterpret_cast<R*>(base + off); off += al(3 * (size_t)Tx * Ty * sizeof(R));
    R* Qs = reinterpret_cast<R*>(base + off); off += al(3 * (size_t)Tx * Ty * sizeof(R));
    R* Zs = reinterpret_cast<R*>(base + off); off += al(3 * (size_t)zplane * sizeof(R));
    R* F1s = reinterpret_cast<R*>(base + off); off += al((size_t)BW * BH * sizeof(R));
    R* F2s = reinterpret_cast<R*>(base + off); off += al((size_t)BW * BH * sizeof(R));
    R* ALs = reinterpret_cast<R*>(base + off);

    const CUtensorMap* tm = P.tmaps + (size_t)pair * TM_PER_PAIR;
    if (threadIdx.x == 0) {
        sh_fail = 0;
        mbar_init(bar, 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned bytes = (unsigned)(2 * (size_t)BW * BH + 2 * (size_t)BW * (BH - 1) + 3 * (size_t)Tx * Ty) * sizeof(R);
        if (need_q) bytes += (unsigned)(3 * (size_t)Tx * Ty * sizeof(R));
        mbar_expect_tx(bar, bytes);
        tma_load_2d(F1s, tm + TM_F1, xs, ys, bar);
        tma_load_2d(F2s, tm + TM_F2, xs, ys, bar);
        tma_load_2d(ALs, tm + TM_AL, 2 * xs, ys, bar);
        tma_load_3d(Rs, tm + TM_R, x0, y0, 0, bar);
        if (need_q) tma_load_3d(Qs, tm + TM_Q, x0, y0, 0, bar);
    }
    // zero the local solution (and its ring) while the copies are in flight
    for (int i = threadIdx.x; i < 3 * zplane; i += NT) Zs[i] = R(0);
    if (threadIdx.x == 0) {
        if (!mbar_wait_bounded(bar, P.spin_limit)) {
            sh_fail = 1;
            atomicOr(P.err, 1);
            mbar_wait_bounded(bar, P.spin_limit);  // give copies in flight a last chance to land
        }
    }
    __syncthreads();
    if (sh_fail) return;
    // every thread observes the completed phase (visibility of the async copies)
    if (!mbar_wait_bounded(bar, P.spin_limit)) atomicOr(P.err, 1);

    // r <- r - a q on the owned tile; write r back; partial r.r
    const R a = need_q ? (R)P.sc[pair].a : R(0);
    R* rg = reinterpret_cast<R*>(P.r) + pd.vec_off;
    R rr = R(0);  // per-thread partials in the working precision, FP64 across threads
    const int ntile = tw * th;
    for (int k = threadIdx.x; k < ntile; k += NT) {
        const int j = k / tw, i = k - j * tw;
        const int si = j * Tx + i;
        R v0 = Rs[si], v1 = Rs[si + Tx * Ty], v2 = Rs[si + 2 * Tx * Ty];
        if (need_q) {
            v0 = v0 - a * Qs[si];
            v1 = v1 - a * Qs[si + Tx * Ty];
            v2 = v2 - a * Qs[si + 2 * Tx * Ty];
            Rs[si] = v0; Rs[si + Tx * Ty] = v1; Rs[si + 2 * Tx * Ty] = v2;
            const long long o = (long long)(y0 + j) * pitch + (x0 + i);
            rg[o] = v0; rg[o + plane] = v1; rg[o + 2 * plane] = v2;
        }
        rr += v0 * v0 + v1 * v1 + v2 * v2;
    }
    __syncthreads();

    // local solve on the extended tile
    const int ex0 = max(x0 - ov, 0), ex1 = min(x0 + tw + ov, W);
    const int ey0 = max(y0 - ov, 0), ey1 = min(y0 + th + ov, H);
    const int Ew = ex1 - ex0, Eh = ey1 - ey0;
    const R lam = (R)P.lam;
    const int ncol = (P.sweeps > 0) ? 1 + 4 * P.sweeps : 1;
    for (int step = 0; step < ncol; ++step) {
        int col = -1;  // -1: every node at once (block Jacobi)
        if (P.sweeps > 0) {
            const int m = step % 4;  // 0,1,2,1 repeating, then the final 0
            col = (m == 0) ? 0 : (m == 1 ? 1 : (m == 2 ? 2 : 1));
        }
        const int M = (col < 0) ? Ew : (Ew + 2) / 3;
        const int nwork = M * Eh;
        for (int k = threadIdx.x; k < nwork; k += NT) {
            const int j = k / M, m = k - j * M;
            int i;
            if (col < 0) i = m;
            else {
                const int base = ((col - (ex0 + ey0 + j)) % 3 + 3) % 3;
                i = base + 3 * m;
                if (i >= Ew) continue;
            }
            const int gx = ex0 + i, gy = ey0 + j;
            R r0 = R(0), r1 = R(0), r2 = R(0);
            if (gx >= x0 && gx < x0 + tw && gy >= y0 && gy < y0 + th) {
                const int si = (gy - y0) * Tx + (gx - x0);
                r0 = Rs[si]; r1 = Rs[si + Tx * Ty]; r2 = Rs[si + 2 * Tx * Ty];
            }
            const int ci = (gy - ys) * BW + (gx - xs);
            const int zi = (gy - (y0 - ov) + 1) * ZW + (gx - (x0 - ov) + 1);
            node_update<R>(gx, gy, W, H, F1s, F2s, ALs, ci, BW, Zs, zi, ZW, zplane, r0, r1, r2, lam);
        }
        __syncthreads();
    }

    // write the owned part of z; partial r.z
    R* zg = reinterpret_cast<R*>(P.z) + pd.vec_off;
    R rz = R(0);
    for (int k = threadIdx.x; k < ntile; k += NT) {
        const int j = k / tw, i = k - j * tw;
        const int si = j * Tx + i;
        const int zi = (y0 + j - (y0 - ov) + 1) * ZW + (x0 + i - (x0 - ov) + 1);
        const R v0 = Zs[zi], v1 = Zs[zi + zplane], v2 = Zs[zi + 2 * zplane];
        const long long o = (long long)(y0 + j) * pitch + (x0 + i);
        zg[o] = v0; zg[o + plane] = v1; zg[o + 2 * plane] = v2;
        rz += Rs[si] * v0 + Rs[si + Tx * Ty] * v1 + Rs[si + 2 * Tx * Ty] * v2;
    }
    if (P.apply_only) return;

    const double s_rr = block_sum<NT>((double)rr, sh_red);
    const double s_rz = block_sum<NT>((double)rz, sh_red);
    if (threadIdx.x == 0) {
        P.partial[2 * (long long)ti.w] = s_rr;
        P.partial[2 * (long long)ti.w + 1] = s_rz;
    }
    const int ntiles = pd.tiles_x * pd.tiles_y;
    if (!arrive_last(&P.counter[pair], (unsigned)ntiles, &sh_last)) return;
    const double t_rr = ordered_sum<NT>(P.partial + 2 * (long long)pd.tile0, ntiles, 2, sh_red);
    const double t_rz = ordered_sum<NT>(P.partial + 2 * (long long)pd.tile0 + 1, ntiles, 2, sh_red);
    if (threadIdx.x == 0) {
        PairScalars* s = P.sc + pair;
        if (P.first) {
            s->rz = t_rz;
            s->rr = t_rr;
            s->beta = 0.0;
            if (!isfinite(t_rr) || !isfinite(t_rz)) { s->status = 6; s->done = 1; }
            else if (t_rr <= s->tol2 || t_rr == 0.0) { s->done = 1; }
            else if (!(t_rz > 0.0)) { s->status = 6; s->done = 1; }
        } else {
            s->beta = t_rz / s->rz;
            s->rz = t_rz;
            s->rr = t_rr;
            s->it += 1;
            s->it_total += 1;
            if (!isfinite(t_rr) || !isfinite(t_rz)) { s->status = 6; s->done = 1; }
            else if (t_rr <= s->tol2) { s->done = 1; }
            else if (!(t_rz > 0.0)) { s->status = 6; s->done = 1; }
            else if (s->it >= s->max_it) { s->status = 5; s->done = 1; }
        }
        __threadfence();
        P.counter[pair] = 0u;
    }
}

}  // namespace ofk
