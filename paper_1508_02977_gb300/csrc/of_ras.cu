// The paper's Schwarz method as a stationary iteration (Section 3.2,
// Eq. schwarz): every subdomain solves its extended problem with Dirichlet
// data from the previous global iterate outside it (the transmission
// condition on Gamma_ij), and each node takes its new value from the
// subdomain that owns it (the restricted form).  In correction form,
//   U^k = U^{k-1} + sum_i R~_i^T A_i^{-1} R_i (b - A U^{k-1}),
// R_i the restriction to the extended tile i, R~_i to its owned tile,
// A_i = R_i A R_i^T.  The residual comes from the solver's residual kernel
// (FP64 or double-float, which also folds the correction into U); this file
// holds the local solves: one CTA per subdomain, the element records of the
// extended tile and a one-node ring of zeros in shared memory, and `sweeps`
// symmetric 3-colour block SOR sweeps from zero on the extended tile (the
// preconditioner's local solver, with the right-hand side on every node of
// the extended tile instead of the owned ones only); many sweeps give the
// exact local solve A_i^{-1}.
#include <cuda_runtime.h>

#include "of_launch.h"
#include "of_schwarz.cuh"

namespace ofk {

struct RasParams {
    const PairDesc* pairs;
    const int4* tiles;
    const uint32_t* ntab;      // node table of the grid's extended tile (see schwarz_node_table)
    const void* cell0;         // element records [H][pitch] (storage type of the preconditioner)
    const void* cell1;
    const void* r;             // residual b - A U^{k-1} (inner vectors, storage precision)
    void* d;                   // out: owned part of the local corrections
    const PairScalars* sc;     // a pair with done set contributes d = 0
    double* partial;           // [ntiles]: ||d||^2 of the owned tile
    int* err;                  // device error word (index checks of the bounds-check build)
    double lam, omega;
    int Tx, Ty, ov, sweeps;
};

template <typename R, int NPT>
__global__ void __launch_bounds__(sch_max_threads(sizeof(R) == 8), 1) k_ras(const RasParams P) {
    using Rec = typename CellT<R>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ double sh_red[32];
    const int NT = blockDim.x;
    const int4 ti = P.tiles[blockIdx.x];
    const PairDesc pd = P.pairs[ti.x];
    const int W = pd.W, H = pd.H, pitch = pd.pitch;
    const int Tx = P.Tx, Ty = P.Ty, ov = P.ov;
    const int RW = sch_rw(Tx, ov), RH = sch_rh(Ty, ov), nc = RW * RH, cpad = sch_cpad(ov);
    const int x0 = ti.y * Tx, y0 = ti.z * Ty;
    const int tw = min(Tx, W - x0), th = min(Ty, H - y0);
    const int ex0 = max(x0 - ov, 0), ex1 = min(x0 + tw + ov, W);
    const int ey0 = max(y0 - ov, 0), ey1 = min(y0 + th + ov, H);
    const long long plane = (long long)H * pitch;
    const R* r = static_cast<const R*>(P.r) + pd.vec_off;
    R* d = static_cast<R*>(P.d) + pd.vec_off;
    const bool skip = P.sc[ti.x].done != 0;

    Rec* C0 = reinterpret_cast<Rec*>(smem);
    Rec* C1 = C0 + nc;
    R* Zs = reinterpret_cast<R*>(C1 + nc);
    // element records of the window (zero outside the image: missing
    // triangles add nothing); z = 0 everywhere, including the ring
    const Rec* g0 = static_cast<const Rec*>(P.cell0) + pd.frame_off;
    const Rec* g1 = static_cast<const Rec*>(P.cell1) + pd.frame_off;
    for (int i = threadIdx.x; i < nc; i += NT) {
        const int cx = x0 - cpad + i % RW, cy = y0 - ov - 1 + i / RW;
        Rec a{}, b{};
        if (!skip && cx >= 0 && cx < W && cy >= 0 && cy < H && OF_CHECK(P.err, (long long)cy * pitch + cx, plane)) {
            a = g0[(long long)cy * pitch + cx];
            b = g1[(long long)cy * pitch + cx];
        }
        C0[i] = a;
        C1[i] = b;
    }
    for (int i = threadIdx.x; i < 3 * nc; i += NT) Zs[i] = R(0);
    __syncthreads();

    CellView<R> C;
    C.c0 = C0;
    C.c1 = C1;
    const R hl = R(0.5) * (R)P.lam;
    const R om = (R)P.omega;
    NodeState<R> ns[3][NPT];
#pragma unroll
    for (int col = 0; col < 3; ++col) {
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            const uint32_t e = P.ntab[(col * NPT + k) * NT + threadIdx.x];
            NodeState<R>& n = ns[col][k];
            n.c = -1;
            n.b0 = n.b1 = n.b2 = R(0);
            n.B = Blk<R>{R(0), R(0), R(0), R(0), R(0), R(0)};
            if (skip || e == 0xffffffffu) continue;
            const int li = (int)(e & 0xffffu), lj = (int)(e >> 16);
            const int gx = x0 - ov + li, gy = y0 - ov + lj;
            const int c = (lj + 1) * RW + (li + cpad - ov);
            if (gx < ex0 || gx >= ex1 || gy < ey0 || gy >= ey1) continue;  // clipped: stays 0
            if (!OF_CHECK(P.err, c - RW - 1, nc) || !OF_CHECK(P.err, c + RW + 1, nc) ||
                !OF_CHECK(P.err, (long long)gy * pitch + gx, plane))
                continue;
            const int vc = (gx < W - 1 && gy < H - 1), vsw = (gx >= 1 && gy >= 1);
            const int vw = (gx >= 1 && gy < H - 1), vs = (gx < W - 1 && gy >= 1);
            const int nE = vc + vs, nN = vc + vw, nW = vsw + vw, nS = vsw + vs;
            n.c = c | (nE << 24) | (nN << 26) | (nW << 28) | (nS << 30);
            node_block<R>(C, c, RW, hl * R(nE), hl * R(nN), hl * R(nW), hl * R(nS), n.B);
            // R_i r: the residual on every node of the extended tile
            const long long o = (long long)gy * pitch + gx;
            n.b0 = r[o];
            n.b1 = r[o + plane];
            n.b2 = r[o + 2 * plane];
            if (col == 0) node_jacobi<R>(Zs, nc, n, P.sweeps > 0 ? om : R(1));
        }
    }
    __syncthreads();
    ZOut<R> none{};
#define OF_RSTEP(col, FRESH)                                                        \
    {                                                                               \
        _Pragma("unroll") for (int k = 0; k < NPT; ++k)                             \
            node_step<R, FRESH, false>(C, Zs, nc, RW, hl, om, ns[col][k], none);    \
        __syncthreads();                                                            \
    }
    // colour order 0,1,2,1 per sweep, then 0 (the first 0 was the Jacobi step)
    if (P.sweeps == 0) {
#pragma unroll
        for (int col = 1; col < 3; ++col)
#pragma unroll
            for (int k = 0; k < NPT; ++k) node_jacobi<R>(Zs, nc, ns[col][k]);
        __syncthreads();
    } else {
#pragma unroll
        for (int k = 0; k < NPT; ++k) node_step_first1<R>(C, Zs, nc, RW, hl, om, ns[1][k]);
        __syncthreads();
        OF_RSTEP(2, true)
        OF_RSTEP(1, false)
        for (int sw = 1; sw < P.sweeps; ++sw) {
            OF_RSTEP(0, false)
            OF_RSTEP(1, false)
            OF_RSTEP(2, false)
            OF_RSTEP(1, false)
        }
        OF_RSTEP(0, false)
    }
#undef OF_RSTEP
    // owned part of the local solution -> d (zero for a finished pair)
    double s2 = 0.0;
    for (int i = threadIdx.x; i < tw * th; i += NT) {
        const int gx = x0 + i % tw, gy = y0 + i / tw;
        const int c = (gy - y0 + ov + 1) * RW + (gx - x0 + cpad);
        const long long o = (long long)gy * pitch + gx;
        if (!OF_CHECK(P.err, o, plane) || !OF_CHECK(P.err, c, nc)) continue;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const R v = skip ? R(0) : Zs[c + k * nc];
            d[o + k * plane] = v;
            s2 += (double)v * (double)v;
        }
    }
    const double t = block_sum_rt(s2, sh_red);
    if (threadIdx.x == 0) P.partial[ti.w] = t;
}

// Per pair: ||U^k - U^{k-1}||_2 from the tile partials (fixed order) into
// hist[pair]; prepares the next residual launch to fold d into U (a = 0, so
// that the correction is exactly d) and counts the iteration.
__global__ void k_ras_finish(const PairDesc* pairs, PairScalars* sc, const double* partial, double* hist) {
    __shared__ double sh_red[32];
    const int pair = blockIdx.x;
    const PairDesc pd = pairs[pair];
    const int nt = pd.tiles_x * pd.tiles_y;
    const double s = ordered_sum_rt(partial + pd.tile0, nt, 1, sh_red);
    if (threadIdx.x == 0) {
        PairScalars* p = sc + pair;
        const bool active = !p->done;
        hist[pair] = active ? sqrt(s) : 0.0;
        p->a = 0.0;
        p->it = 1;
        if (active) p->it_total += 1;
    }
}

}  // namespace ofk

namespace ofl {

using namespace ofk;

size_t ras_smem_bytes(int fp64, int Tx, int Ty, int ov) {
    const size_t nc = (size_t)sch_rw(Tx, ov) * sch_rh(Ty, ov);
    return fp64 ? nc * (2 * cell_bytes<double>() + 3 * sizeof(double))
                : nc * (2 * cell_bytes<float>() + 3 * sizeof(float));
}

template <typename R, int NPT>
static cudaError_t ras_t(const SolveBufs& B, const void* c0, const void* c1, double* hist, cudaStream_t st) {
    RasParams P;
    P.pairs = B.pairs;
    P.tiles = B.tiles;
    P.ntab = B.ntab;
    P.cell0 = c0;
    P.cell1 = c1;
    P.r = B.r;
    P.d = B.d;
    P.sc = B.sc;
    P.partial = B.partS;
    P.err = B.err;
    P.lam = B.lam;
    P.omega = B.omega;
    P.Tx = B.Tx;
    P.Ty = B.Ty;
    P.ov = B.ov;
    P.sweeps = B.sweeps;
    const size_t smem = ras_smem_bytes(sizeof(R) == 8, B.Tx, B.Ty, B.ov);
    cudaError_t e = cudaFuncSetAttribute(k_ras<R, NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_ras<R, NPT><<<B.ntiles, B.sch_threads, smem, st>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ras_finish<<<B.npairs, 256, 0, st>>>(B.pairs, B.sc, B.partS, hist);
    return cudaGetLastError();
}

cudaError_t launch_ras(const SolveBufs& B, const void* c0, const void* c1, double* hist, cudaStream_t st) {
    if (B.fp64) return B.sch_npt == 1 ? ras_t<double, 1>(B, c0, c1, hist, st) : ras_t<double, 2>(B, c0, c1, hist, st);
    return B.sch_npt == 1 ? ras_t<float, 1>(B, c0, c1, hist, st) : ras_t<float, 2>(B, c0, c1, hist, st);
}

}  // namespace ofl
