// Coarse correction of the two-level preconditioner:
//   z = M_1 r + R_0^T A_0^{-1} R_0 r,   A_0 = R_0 A R_0^T,
// M_1 the restricted Schwarz sweeps (of_schwarz.cuh) and R_0 the bilinear
// hat functions of a coarse grid (nodes at x = 0, s, 2s, ... and W - 1, the
// same in y), one per component.  With the coarse space the iteration count
// stops growing with the number of subdomains and stays low on smooth data
// (K_sigma pre-smoothing), where the one-level method loses most.
//
// A_0 is assembled per solve, one CTA per coarse cell, from the element
// matrices of Section 2.2 (the same P1 data term and stiffness as the fine
// operator).  Coarse unknowns are ordered node by node (u = 3 node + c), so
// A_0 is banded with half bandwidth b = 3 nx + 5; one CTA factors it
// (band Cholesky over a sliding window in shared memory) and one warp per
// column forms the dense inverse by forward and backward substitution.
// Each application is a restriction, one dense product with the inverse and
// a bilinear prolongation.
// All sums run in a fixed order: the results do not depend on scheduling.
#include <cuda_runtime.h>

#include <algorithm>

#include "of_common.cuh"
#include "of_launch.h"
#include "of_schwarz.cuh"

namespace ofl {

using namespace ofk;

constexpr size_t kMaxSmem = 227 * 1024;  // opt-in shared memory per CTA

// hat weights of node (x, y) inside cell [x0, x1] x [y0, y1]: corners
// a = 0 (x0, y0), 1 (x1, y0), 2 (x0, y1), 3 (x1, y1)
template <typename R>
__device__ __forceinline__ void cell_hats(int x, int y, const CoarseCell& c, R ph[4]) {
    const R wx = R(x - c.x0) / R(c.x1 - c.x0), wy = R(y - c.y0) / R(c.y1 - c.y0);
    ph[0] = (R(1) - wx) * (R(1) - wy);
    ph[1] = wx * (R(1) - wy);
    ph[2] = (R(1) - wx) * wy;
    ph[3] = wx * wy;
}

// node range of a cell: x0 <= x < x1 (x <= x1 for the last cell), same in y,
// so that every fine node belongs to exactly one cell
__device__ __forceinline__ void cell_nodes(const CoarseCell& c, const CoarsePair& cp, int& nx, int& ny) {
    nx = c.x1 - c.x0 + (c.k == cp.nx - 2 ? 1 : 0);
    ny = c.y1 - c.y0 + (c.l == cp.ny - 2 ? 1 : 0);
}

// Block sum of NV values per thread into out[0..NV) (fixed order).
template <typename R, int NV>
__device__ __forceinline__ void block_sum_vec(R (&v)[NV], R* sh, R* out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0)
        for (int i = 0; i < NV; ++i) sh[w * NV + i] = v[i];
    __syncthreads();
    for (int i = threadIdx.x; i < NV; i += blockDim.x) {
        R t = R(0);
        for (int j = 0; j < nw; ++j) t += sh[j * NV + i];
        out[i] = t;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- A_0 --
// One CTA per coarse cell: the 12 x 12 block of the cell (4 corners x 3
// components, index 3 a + c), upper triangle accumulated per thread.
template <typename R>
__global__ void __launch_bounds__(256) k_coarse_assemble(const PairDesc* pairs, const CoarsePair* cps,
                                                         const CoarseCell* cells, const R* __restrict__ f1a,
                                                         const R* __restrict__ f2a, const R* __restrict__ ala,
                                                         double lam_d, double gms_d, R* __restrict__ blk) {
    constexpr int NU = 78;  // 12 * 13 / 2
    __shared__ R sh[8 * NU];
    __shared__ R res[NU];
    const CoarseCell c = cells[blockIdx.x];
    const PairDesc pd = pairs[c.pair];
    const int pitch = pd.pitch;
    const R* f1 = f1a + pd.frame_off;
    const R* f2 = f2a + pd.frame_off;
    const R* al = ala + 2 * pd.frame_off;
    const R lam = (R)lam_d, gms = (R)gms_d, third = R(1) / R(3), k12 = R(0.5) / R(12), kA = R(0.5);
    R acc[NU];
#pragma unroll
    for (int i = 0; i < NU; ++i) acc[i] = R(0);
    // squares with their lower-left node in [x0, x1) x [y0, y1): inside the cell
    const int sw = c.x1 - c.x0, sh_ = c.y1 - c.y0;
    for (int i = threadIdx.x; i < sw * sh_; i += blockDim.x) {
        const int x = c.x0 + i % sw, y = c.y0 + i / sw;
        const long long o = (long long)y * pitch + x;
        // corners A=(x,y) B=(x+1,y) C=(x+1,y+1) D=(x,y+1)
        R hA[4], hB[4], hC[4], hD[4];
        cell_hats<R>(x, y, c, hA);
        cell_hats<R>(x + 1, y, c, hB);
        cell_hats<R>(x + 1, y + 1, c, hC);
        cell_hats<R>(x, y + 1, c, hD);
        const R a2 = f2[o], b2 = f2[o + 1], c2 = f2[o + pitch + 1], d2 = f2[o + pitch];
        const R a1 = f1[o], b1 = f1[o + 1], c1 = f1[o + pitch + 1], d1 = f1[o + pitch];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            // vertices (A, B, C) or (A, D, C); g and the P1 gradients of the hats
            const R* hM = t == 0 ? hB : hD;
            R g[3];
            if (t == 0) { g[0] = b2 - a2; g[1] = c2 - b2; g[2] = -(a1 + b1 + c1) * third * gms; }
            else        { g[0] = c2 - d2; g[1] = d2 - a2; g[2] = -(a1 + d1 + c1) * third * gms; }
            const R alpha = al[2 * o + t];
            const R Lc[3] = {alpha, alpha, lam};
            R S[4], gx[4], gy[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                S[a] = hA[a] + hM[a] + hC[a];
                if (t == 0) { gx[a] = hB[a] - hA[a]; gy[a] = hC[a] - hB[a]; }
                else        { gx[a] = hC[a] - hD[a]; gy[a] = hD[a] - hA[a]; }
            }
            int idx = 0;
#pragma unroll
            for (int p = 0; p < 12; ++p) {
#pragma unroll
                for (int q = p; q < 12; ++q) {
                    const int a = p / 3, ci = p % 3, b = q / 3, di = q % 3;
                    const R mass = S[a] * S[b] + hA[a] * hA[b] + hM[a] * hM[b] + hC[a] * hC[b];
                    R v = k12 * g[ci] * g[di] * mass;
                    if (ci == di) v += kA * Lc[ci] * (gx[a] * gx[b] + gy[a] * gy[b]);
                    acc[idx++] += v;
                }
            }
        }
    }
    block_sum_vec<R, NU>(acc, sh, res);
    R* out = blk + (long long)blockIdx.x * 144;
    for (int i = threadIdx.x; i < NU; i += blockDim.x) {
        // upper-triangle index i -> (p, q)
        int p = 0, rem = i;
        while (rem >= 12 - p) { rem -= 12 - p; ++p; }
        const int q = p + rem;
        out[p * 12 + q] = res[i];
        out[q * 12 + p] = res[i];
    }
}

// Dense A_0 (column-major, symmetric) of every pair from the cell blocks:
// entry (I, J) sums the blocks of the cells containing both coarse nodes.
template <typename R>
__global__ void k_coarse_scatter(const CoarsePair* cps, int npairs, const R* __restrict__ blk, R* __restrict__ A) {
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // work item: (pair, node I, neighbour offset 0..8, components c, d)
    long long rem = gid;
    int pair = 0;
    for (; pair < npairs; ++pair) {
        const long long n = (long long)cps[pair].nx * cps[pair].ny * 81;
        if (rem < n) break;
        rem -= n;
    }
    if (pair >= npairs) return;
    const CoarsePair cp = cps[pair];
    const int cd = (int)(rem % 9), nb = (int)((rem / 9) % 9);
    const long long node = rem / 81;
    const int k = (int)(node % cp.nx), l = (int)(node / cp.nx);
    const int k2 = k + nb % 3 - 1, l2 = l + nb / 3 - 1;
    if (k2 < 0 || l2 < 0 || k2 >= cp.nx || l2 >= cp.ny) return;
    const int c = cd / 3, d = cd % 3;
    R v = R(0);
    for (int cl = max(max(l, l2) - 1, 0); cl <= min(min(l, l2), cp.ny - 2); ++cl)
        for (int ck = max(max(k, k2) - 1, 0); ck <= min(min(k, k2), cp.nx - 2); ++ck) {
            const int a = (k - ck) + 2 * (l - cl), b = (k2 - ck) + 2 * (l2 - cl);
            v += blk[(long long)(cp.cell0 + cl * (cp.nx - 1) + ck) * 144 + (3 * a + c) * 12 + (3 * b + d)];
        }
    const long long I = 3 * node + c, J = 3 * ((long long)l2 * cp.nx + k2) + d;  // node-major: banded
    A[cp.moff + J * cp.n0 + I] = v;
}

// X <- (X + X^T) / 2: the inverse formed column by column is symmetric only
// up to rounding; the preconditioner needs it exactly symmetric
template <typename R>
__global__ void k_symmetrize(R* __restrict__ A, int n) {
    const int j = blockIdx.y * blockDim.y + threadIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && j < n && i < j) {
        const R v = R(0.5) * (A[(long long)j * n + i] + A[(long long)i * n + j]);
        A[(long long)j * n + i] = v;
        A[(long long)i * n + j] = v;
    }
}

// Band Cholesky A_0 = L L^T of one pair (half bandwidth b), one CTA,
// right-looking over a (b+1) x (b+1) window of the trailing matrix kept in
// shared memory (rows and columns in a ring of b+1 slots).  L is written
// twice: by rows (Lr[i][i-j], j = i-b..i) for the forward substitution and
// by columns (Lc[j][i-j], i = j..j+b) for the backward one.  The row that
// enters the window at each step is read from the symmetric matrix's column
// (contiguous) one step ahead.  info: 0, or the 1-based index of a
// non-positive pivot.
template <typename R>
__global__ void __launch_bounds__(1024) k_band_cholesky(const CoarsePair* cps, int pair, int b, const R* __restrict__ A,
                                                        R* __restrict__ Lr, R* __restrict__ Lc, int* info) {
    extern __shared__ __align__(16) unsigned char wsm[];
    const int w = b + 1;
    R* Wn = reinterpret_cast<R*>(wsm);      // [w][w] window, lower part used
    R* v = Wn + (size_t)w * w;              // [w] scaled column
    __shared__ int bad;
    const CoarsePair cp = cps[pair];
    const int n = cp.n0;
    const R* Ap = A + cp.moff;
    R* Lrp = Lr + cp.boff;
    R* Lcp = Lc + cp.boff;
    if (threadIdx.x == 0) bad = 0;
    for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
        const int i = t / w, k = t % w;
        Wn[i * w + k] = (i < n && k < n && k <= i) ? Ap[(long long)i * n + k] : R(0);
    }
    // entering row of step j: row j + w, columns j+1 .. j+w = column j + w,
    // rows j+1 .. j+w of the symmetric matrix
    auto fetch = [&](int j) -> R {
        const int ni = j + w, k = j + 1 + (int)threadIdx.x;
        return (threadIdx.x < (unsigned)w && ni < n) ? Ap[(long long)ni * n + k] : R(0);
    };
    R nxt = fetch(0);
    __syncthreads();
    const int ua = 1 + ((int)threadIdx.x >> 3), t8 = (int)threadIdx.x & 7;
    int sj = 0;  // j mod w
    for (int j = 0; j < n; ++j) {
        const R d = Wn[sj * w + sj];
        if (!(d > R(0))) {
            if (threadIdx.x == 0) { bad = j + 1; info[pair] = j + 1; }
            __syncthreads();
            break;
        }
        const R ljj = sqrt(d);
        const int m = min(b, n - 1 - j);  // rows below the diagonal inside the band
        if ((int)threadIdx.x <= m) {
            const int t = threadIdx.x, i = j + t;
            int si = sj + t;
            if (si >= w) si -= w;
            const R lij = (t == 0) ? ljj : Wn[si * w + sj] / ljj;
            v[t] = lij;
            Lrp[(long long)i * w + t] = lij;
            Lcp[(long long)j * w + t] = lij;
        }
        const R cur = nxt;
        if (j + 1 < n) nxt = fetch(j + 1);
        __syncthreads();
        // slot sj (row j, no longer read) takes row j + w: columns j+1 .. j+w; the
        // update below touches rows j+1 .. j+m only
        if ((int)threadIdx.x < w) {
            int rc = sj + 1 + (int)threadIdx.x;
            if (rc >= w) rc -= w;
            Wn[sj * w + rc] = cur;
        }
        for (int a = ua; a <= m; a += (int)(blockDim.x >> 3)) {
            int ra = sj + a;
            if (ra >= w) ra -= w;
            const R va = v[a];
            for (int c = 1 + t8; c <= a; c += 8) {
                int rc = sj + c;
                if (rc >= w) rc -= w;
                Wn[ra * w + rc] -= va * v[c];
            }
        }
        __syncthreads();
        if (++sj == w) sj = 0;
    }
    if (threadIdx.x == 0 && !bad) info[pair] = 0;
}

// Blocked band Cholesky (right-looking, panels of CB_NB = 32 columns), used
// whenever its window fits in shared memory.  The window W holds rows and
// columns J .. J+S-1 (S = 32 + b rounded up to 4) at slots g mod S (row
// stride S + 1: column reads are free of bank conflicts).  Per panel
// J .. J+31, held as P[k][r] = entry (J + r, J + k):
//  1. warp 0 factors the 32 x 32 diagonal block (a pivot, a scaled column
//     and a rank-1 update per column, lane r = row r); then every row below
//     it solves against that block (L21 = A21 L11^{-T}) on its own;
//  2. the L entries are written out (column band layout; the row layout is
//     filled from it afterwards by k_band_rows);
//  3. rank-32 update of the trailing b x b triangle, one 4 x 4 tile of
//     products per thread; then the 32 rows that enter the window (read from
//     the symmetric matrix at the start of the panel) are stored.
// Shared-memory read-modify-write loops load a chunk of 8 before they store
// it (the compiler cannot move a load above a store to the same array) and
// are not unrolled further: fully unrolled panels overflow the instruction
// cache, and register rows with compare-and-select indexing were slower.
constexpr int CB_NB = 32;
constexpr int CB_EN = 12;     // entering-row values per thread
constexpr int CB_MAXT = 640;  // threads (launch bound): 32 S <= CB_EN CB_MAXT for S <= 224
__host__ __device__ constexpr int cb_window(int b) { return CB_NB + ((b + 3) / 4) * 4; }
__host__ __device__ constexpr long long cb_smem_elems(int b) {
    return (long long)cb_window(b) * (cb_window(b) + 1) + (long long)CB_NB * cb_window(b) + 1;
}
static int cb_threads(int b) {
    const int S = cb_window(b), tb = (b + 3) / 4;
    int t = std::max(std::max(tb * (tb + 1) / 2, S), (CB_NB * S + CB_EN - 1) / CB_EN);
    t = (t + 31) / 32 * 32;
    return std::min(t, CB_MAXT);
}

template <typename R>
__device__ __forceinline__ void load4(const R* p, R (&v)[4]) {
    if constexpr (sizeof(R) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        v[0] = p[0]; v[1] = p[1]; v[2] = p[2]; v[3] = p[3];
    }
}

template <typename R>
__global__ void __launch_bounds__(CB_MAXT) k_band_cholesky_blk(const CoarsePair* cps, int pair, int b,
                                                               const R* __restrict__ A, R* __restrict__ Lc,
                                                               int* info) {
    extern __shared__ __align__(16) unsigned char csm[];
    const int S = cb_window(b), S1 = S + 1, w = b + 1, tb = (b + 3) / 4, ntiles = tb * (tb + 1) / 2;
    R* P = reinterpret_cast<R*>(csm);  // [CB_NB][S] (first: 16-byte aligned rows)
    R* W = P + (size_t)CB_NB * S;      // [S][S + 1]
    R* flag = W + (size_t)S * S1;      // [1]: failure
    const CoarsePair cp = cps[pair];
    const int n = cp.n0;
    const R* Ap = A + cp.moff;
    R* Lcp = Lc + cp.boff;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31;
    for (int e = tid; e < S * S; e += nth) {
        const int r = e / S, c = e - r * S;
        W[r * S1 + c] = (r < n && c <= r && r - c <= b) ? Ap[(long long)r * n + c] : R(0);
    }
    __syncthreads();
    int failed = 0;
    for (int J = 0; J < n; J += CB_NB) {
        const int nb = min(CB_NB, n - J);
        const int base = J % S;
        // the rows entering the window after this panel (g = J + S + q, columns
        // J + 32 .. J + 32 + S - 1): loaded first, stored after the update
        R ent[CB_EN];
#pragma unroll
        for (int k = 0; k < CB_EN; ++k) {
            const int e = tid + k * nth;
            ent[k] = R(0);
            if (e < CB_NB * S) {
                const int q = e / S, c = e - q * S;
                const int g = J + S + q, cg = J + CB_NB + c;
                if (g < n && cg <= g && g - cg <= b) ent[k] = Ap[(long long)g * n + cg];
            }
        }
        // panel into P: P[k][r] = entry (J + r, J + k), zero outside the band and the matrix
        for (int e = tid; e < CB_NB * S; e += nth) {
            const int k = e / S, r = e - k * S;
            int sr = base + r, sk = base + k;
            if (sr >= S) sr -= S;
            if (sk >= S) sk -= S;
            P[e] = (k < nb && k <= r && J + r < n) ? W[sr * S1 + sk] : R(0);
        }
        __syncthreads();
        // 1a. diagonal block, warp 0 (lane r = row r)
        if (tid < 32) {
            const int r = lane;
            int badj = 0;
            for (int jj = 0; jj < nb; ++jj) {
                const R d = P[jj * S + jj];
                if (!(d > R(0)) && !badj) badj = jj + 1;
                const R l = d > R(0) ? sqrt(d) : R(1);
                __syncwarp();
                if (r == jj) P[jj * S + jj] = l;
                else if (r > jj) P[jj * S + r] = P[jj * S + r] / l;
                __syncwarp();
                if (r > jj) {
                    const R cj = P[jj * S + r];
                    const int kmax = min(r, nb - 1);
                    for (int k0 = jj + 1; k0 <= kmax; k0 += 8) {
                        R a[8], q[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (k0 + u <= kmax) { a[u] = P[(k0 + u) * S + r]; q[u] = P[jj * S + k0 + u]; }
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (k0 + u <= kmax) P[(k0 + u) * S + r] = a[u] - cj * q[u];
                    }
                }
                __syncwarp();
            }
            if (lane == 0) flag[0] = (R)badj;
        }
        __syncthreads();
        if (flag[0] != R(0)) {  // uniform
            failed = J + (int)flag[0];
            break;
        }
        // 1b. rows below the block, one per thread, column by column
        for (int r = CB_NB + tid; r < S; r += nth) {
            if (J + r >= n) continue;
            for (int k = 0; k < nb; ++k) {
                const R x = P[k * S + r] / P[k * S + k];
                P[k * S + r] = x;
                for (int m0 = k + 1; m0 < nb; m0 += 8) {
                    R a[8], q[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (m0 + u < nb) { a[u] = P[(m0 + u) * S + r]; q[u] = P[k * S + m0 + u]; }
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (m0 + u < nb) P[(m0 + u) * S + r] = a[u] - x * q[u];
                }
            }
        }
        __syncthreads();
        // 2. L out: entry (J + r, J + k), r - k <= b
        for (int k = tid >> 5; k < nb; k += nth >> 5)
            for (int r = k + lane; r < S && r - k <= b && J + r < n; r += 32)
                Lcp[(long long)(J + k) * w + (r - k)] = P[k * S + r];
        // 3. trailing update of window rows/columns 32 .. S-1 (only when rows remain)
        if (J + nb < n) {
            for (int t = tid; t < ntiles; t += nth) {
                int I = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
                while (I * (I + 1) / 2 > t) --I;
                while ((I + 1) * (I + 2) / 2 <= t) ++I;
                const int Jt = t - I * (I + 1) / 2;
                const int r0 = CB_NB + 4 * I, c0 = CB_NB + 4 * Jt;
                R acc[4][4];
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) acc[x][y] = R(0);
#pragma unroll 4
                for (int k = 0; k < CB_NB; ++k) {
                    R av[4], bv[4];
                    load4<R>(P + k * S + r0, av);
                    load4<R>(P + k * S + c0, bv);
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] += av[x] * bv[y];
                }
                int sc = base + c0;
                if (sc >= S) sc -= S;
                int ro[4];
                R old[4][4];
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    int sx = base + r0 + x;
                    if (sx >= S) sx -= S;
                    ro[x] = sx * S1 + sc;
#pragma unroll
                    for (int y = 0; y < 4; ++y) old[x][y] = W[ro[x] + y];
                }
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) W[ro[x] + y] = old[x][y] - acc[x][y];
            }
        }
        // entering rows take the slots of rows J .. J+31
#pragma unroll
        for (int k = 0; k < CB_EN; ++k) {
            const int e = tid + k * nth;
            if (e < CB_NB * S) {
                const int q = e / S, c = e - q * S;
                int sg = base + q, sc = base + CB_NB + c;
                if (sg >= S) sg -= S;
                if (sc >= S) sc -= S;
                if (sc >= S) sc -= S;
                W[sg * S1 + sc] = ent[k];
            }
        }
        __syncthreads();
    }
    if (tid == 0) info[pair] = failed;
}

// Row band layout from the column one: Lr[i w + t] = L[i][i-t] = Lc[(i-t) w + t].
template <typename R>
__global__ void k_band_rows(const CoarsePair* cps, int pair, int b, const R* __restrict__ Lc, R* __restrict__ Lr) {
    const CoarsePair cp = cps[pair];
    const int w = b + 1;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)cp.n0 * w) return;
    const int i = (int)(e / w), t = (int)(e - (long long)i * w);
    if (i - t >= 0) Lr[cp.boff + e] = Lc[cp.boff + (long long)(i - t) * w + t];
}

// Dense inverse X = A_0^{-1} = L^{-T} L^{-1}, one warp per column i:
// forward L y = e_i, backward L^T x = y, both in blocks of 32 rows (lane t
// <-> row t of the block).  The INV_WARPS columns of a CTA walk the same
// blocks (the forward pass starts at the CTA's first column; rows above a
// column's own index come out as exact zeros), so each block's factor rows
// are staged once per CTA in shared memory by cp.async, one block ahead.
// Per block and column:
//  1. lane t sums the factor entries of its row that reach back before the
//     block against a per-warp ring of the last b + 32 solution values;
//  2. the 32 x 32 triangle inside the block: 31 dependent steps, each a
//     shuffle broadcast of the newly final value and one FMA per lane.
// Row stride of the staged block is a multiple of 32 words: lane t reads its
// row at offsets t + 1 + m (step 1) and t - j (step 2), i.e. 32 distinct banks.
constexpr int INV_WARPS = 8;
__host__ __device__ constexpr int inv_row_stride(int w) { return ((w + 31) / 32) * 32; }
__host__ __device__ constexpr int inv_smem_elems(int b) { return 2 * 32 * inv_row_stride(b + 1) + INV_WARPS * (b + 33); }

template <typename R>
__device__ __forceinline__ void cp_async_el(R* dst, const R* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (sizeof(R) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8 : 0) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}

// stage rows k = R0 + t (forward) or R0 - t (backward), t < nr, entries o <= omax(k)
template <typename R, bool FWD>
__device__ __forceinline__ void inv_stage(R* dst, const R* __restrict__ Lb, int w, int ws, int b, int n, int R0,
                                          int nr) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = warp; t < 32; t += INV_WARPS) {
        const int k = FWD ? R0 + t : R0 - t;
        const int omax = t < nr ? (FWD ? min(b, k) : min(b, n - 1 - k)) : -1;
        for (int o = lane; o < w; o += 32) {
            const bool v = o <= omax;
            cp_async_el<R>(dst + t * ws + o, v ? Lb + (long long)k * w + o : Lb, v);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <typename R>
__global__ void __launch_bounds__(INV_WARPS * 32) k_band_inverse(const CoarsePair* cps, int pair, int b,
                                                                 const R* __restrict__ Lr, const R* __restrict__ Lc,
                                                                 R* __restrict__ X) {
    extern __shared__ __align__(16) unsigned char rsm[];
    const int w = b + 1, ws = inv_row_stride(w), wr = b + 33, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    R* Lbuf = reinterpret_cast<R*>(rsm);                 // [2][32][ws]
    R* ring = Lbuf + 2 * 32 * ws + (size_t)warp * wr;     // y_k at k mod wr
    const CoarsePair cp = cps[pair];
    const int n = cp.n0;
    const int i0 = blockIdx.x * INV_WARPS, i = i0 + warp;
    const bool col = i < n;
    const R* Lrp = Lr + cp.boff;
    const R* Lcp = Lc + cp.boff;
    R* xcol = X + cp.moff + (long long)min(i, n - 1) * n;
    const unsigned full = 0xffffffffu;
    const int t = lane;
    for (int u = lane; u < wr; u += 32) ring[u] = R(0);
    if (col)
        for (int u = lane; u < i0; u += 32) xcol[u] = R(0);
    // ---- forward: row k = R0 + t, L[k][k - o] = Lr[k w + o]
    int pb = i0 % wr;  // ring position of row R0
    int buf = 0;
    inv_stage<R, true>(Lbuf, Lrp, w, ws, b, n, i0, min(32, n - i0));
    for (int R0 = i0; R0 < n; R0 += 32) {
        const int nr = min(32, n - R0);
        if (R0 + 32 < n) inv_stage<R, true>(Lbuf + (buf ^ 1) * 32 * ws, Lrp, w, ws, b, n, R0 + 32, min(32, n - R0 - 32));
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        const R* Lt = Lbuf + buf * 32 * ws + t * ws;  // this lane's row
        R rhs = R(0), invd = R(1);
        if (t < nr) {
            const int omax = min(b, R0 + t);
            R part = R(0);
            int pp = pb - 1;  // ring position of row R0 + t - o for o = t + 1
            if (pp < 0) pp += wr;
            for (int o = t + 1; o <= omax; ++o) {
                part += Lt[o] * ring[pp];
                if (--pp < 0) pp += wr;
            }
            rhs = (R0 + t == i ? R(1) : R(0)) - part;
            invd = R(1) / Lt[0];
        }
        R c[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) c[j] = (t < nr && j < t && t - j <= b) ? Lt[t - j] : R(0);
#pragma unroll
        for (int j = 0; j < 31; ++j) {
            const R yj = __shfl_sync(full, rhs * invd, j);
            if (j < t) rhs -= c[j] * yj;
        }
        const R y = rhs * invd;
        __syncwarp();
        if (t < nr) {
            int pp = pb + t;
            if (pp >= wr) pp -= wr;
            ring[pp] = y;
            if (col) xcol[R0 + t] = y;
        }
        __syncthreads();  // ring and staged block consumed
        pb += 32;
        if (pb >= wr) pb -= wr;
        buf ^= 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    for (int u = lane; u < wr; u += 32) ring[u] = R(0);
    // ---- backward: row k = R0 - t, L[k + o][k] = Lc[k w + o]
    pb = (n - 1) % wr;
    buf = 0;
    __syncthreads();
    inv_stage<R, false>(Lbuf, Lcp, w, ws, b, n, n - 1, min(32, n));
    for (int R0 = n - 1; R0 >= 0; R0 -= 32) {
        const int nr = min(32, R0 + 1);
        if (R0 - 32 >= 0) inv_stage<R, false>(Lbuf + (buf ^ 1) * 32 * ws, Lcp, w, ws, b, n, R0 - 32, min(32, R0 - 31));
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        const R* Lt = Lbuf + buf * 32 * ws + t * ws;
        R rhs = R(0), invd = R(1);
        if (t < nr) {
            const int k = R0 - t, omax = min(b, n - 1 - k);
            R part = R(0);
            int pp = pb - t + t + 1;  // ring position of row k + o for o = t + 1
            if (pp >= wr) pp -= wr;
            for (int o = t + 1; o <= omax; ++o) {
                part += Lt[o] * ring[pp];
                if (++pp >= wr) pp -= wr;
            }
            rhs = (col ? xcol[k] : R(0)) - part;
            invd = R(1) / Lt[0];
        }
        R c[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) c[j] = (t < nr && j < t && t - j <= b) ? Lt[t - j] : R(0);
#pragma unroll
        for (int j = 0; j < 31; ++j) {
            const R xj = __shfl_sync(full, rhs * invd, j);
            if (j < t) rhs -= c[j] * xj;
        }
        const R x = rhs * invd;
        __syncwarp();
        if (t < nr) {
            int pp = pb - t;
            if (pp < 0) pp += wr;
            ring[pp] = x;
            if (col) xcol[R0 - t] = x;
        }
        __syncthreads();
        pb -= 32;
        if (pb < 0) pb += wr;
        buf ^= 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------- application --
// g-partials of a cell: sum over its nodes of hat_a(node) r_c(node).
// One warp per row (rows strided by the warp count), lanes along x; the
// hat factors separate, so a row contributes (1 - wy) S0, (1 - wy) S1,
// wy S0, wy S1 with S0 = sum (1 - wx) r, S1 = sum wx r.
template <typename R>
__global__ void __launch_bounds__(256) k_coarse_restrict(const PairDesc* pairs, const CoarsePair* cps,
                                                         const CoarseCell* cells, const PairScalars* sc,
                                                         int skip_done, int only_pair, const R* __restrict__ ra,
                                                         R* __restrict__ part) {
    __shared__ R sh[8 * 12];
    __shared__ R res[12];
    const CoarseCell c = cells[blockIdx.x];
    if ((skip_done && sc[c.pair].done) || (only_pair >= 0 && c.pair != only_pair)) return;
    const PairDesc pd = pairs[c.pair];
    const CoarsePair cp = cps[c.pair];
    const long long plane = (long long)pd.H * pd.pitch;
    int nx, ny;
    cell_nodes(c, cp, nx, ny);
    const R ix = R(1) / R(c.x1 - c.x0), iy = R(1) / R(c.y1 - c.y0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    R acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = R(0);
    for (int yy = warp; yy < ny; yy += nw) {
        const R* row = ra + pd.vec_off + (long long)(c.y0 + yy) * pd.pitch + c.x0;
        R s0[3] = {R(0), R(0), R(0)}, s1[3] = {R(0), R(0), R(0)};
        for (int x0 = 0; x0 < nx; x0 += 128) {
            R v[4][3];
#pragma unroll
            for (int u = 0; u < 4; ++u) {  // the row's loads first
                const int xx = x0 + lane + 32 * u;
                if (xx < nx) { v[u][0] = row[xx]; v[u][1] = row[xx + plane]; v[u][2] = row[xx + 2 * plane]; }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int xx = x0 + lane + 32 * u;
                if (xx >= nx) continue;
                const R wx = R(xx) * ix;
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    s0[cc] += (R(1) - wx) * v[u][cc];
                    s1[cc] += wx * v[u][cc];
                }
            }
        }
        const R wy = R(yy) * iy;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            acc[cc] += (R(1) - wy) * s0[cc];
            acc[3 + cc] += (R(1) - wy) * s1[cc];
            acc[6 + cc] += wy * s0[cc];
            acc[9 + cc] += wy * s1[cc];
        }
    }
    block_sum_vec<R, 12>(acc, sh, res);
    if (threadIdx.x < 12) part[(long long)blockIdx.x * 12 + threadIdx.x] = res[threadIdx.x];
}

// g = R_0 r from the cell partials: unknown (node (k, l), component c) sums
// the corner partials of the cells around its node in a fixed order
__global__ void k_coarse_gather_f(const CoarseParams P, int total) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= total) return;
    int pi = 0;
    while (pi + 1 < P.npairs && P.cps[pi + 1].voff <= u) ++pi;
    const CoarsePair cp = P.cps[pi];
    if (!((P.apply_only || !P.sc[pi].done) && (P.only_pair < 0 || P.only_pair == pi))) return;
    const int lu = u - cp.voff, c = lu % 3, node = lu / 3, k = node % cp.nx, l = node / cp.nx;
    const float* part = reinterpret_cast<const float*>(P.part);
    float g = 0.f;
    for (int cl = max(l - 1, 0); cl <= min(l, cp.ny - 2); ++cl)
        for (int ck = max(k - 1, 0); ck <= min(k, cp.nx - 2); ++ck)
            g += part[(long long)(cp.cell0 + cl * (cp.nx - 1) + ck) * 12 + 3 * ((k - ck) + 2 * (l - cl)) + c];
    reinterpret_cast<float*>(P.g)[u] = g;
}
__global__ void k_coarse_gather_d(const CoarseParams P, int total) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= total) return;
    int pi = 0;
    while (pi + 1 < P.npairs && P.cps[pi + 1].voff <= u) ++pi;
    const CoarsePair cp = P.cps[pi];
    if (!((P.apply_only || !P.sc[pi].done) && (P.only_pair < 0 || P.only_pair == pi))) return;
    const int lu = u - cp.voff, c = lu % 3, node = lu / 3, k = node % cp.nx, l = node / cp.nx;
    const double* part = reinterpret_cast<const double*>(P.part);
    double g = 0.0;
    for (int cl = max(l - 1, 0); cl <= min(l, cp.ny - 2); ++cl)
        for (int ck = max(k - 1, 0); ck <= min(k, cp.nx - 2); ++ck)
            g += part[(long long)(cp.cell0 + cl * (cp.nx - 1) + ck) * 12 + 3 * ((k - ck) + 2 * (l - cl)) + c];
    reinterpret_cast<double*>(P.g)[u] = g;
}

// y = A_0^{-1} g (one warp per row, g staged in shared memory), g_i y_i per
// row; the last CTA finishes the CG scalars with r.z = (Schwarz's r.z_1) + g.y
template <typename R>
__global__ void __launch_bounds__(256) k_coarse_gemv(const CoarseParams P) {
    extern __shared__ __align__(16) unsigned char gsm[];
    R* gs = reinterpret_cast<R*>(gsm);
    __shared__ double sh_red[32];
    __shared__ int sh_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const R* Ainv = reinterpret_cast<const R*>(P.Ainv);
    R* yv = reinterpret_cast<R*>(P.y);
    for (int pi = 0; pi < P.npairs; ++pi) {
        const CoarsePair cp = P.cps[pi];
        const bool active = (P.apply_only || !P.sc[pi].done) && (P.only_pair < 0 || P.only_pair == pi);
        if (!active) continue;  // uniform over the grid
        const R* gg = reinterpret_cast<const R*>(P.g) + cp.voff;
#pragma unroll 8
        for (int u = threadIdx.x; u < cp.n0; u += blockDim.x) gs[u] = gg[u];
        __syncthreads();
        for (int row = blockIdx.x * nw + warp; row < cp.n0; row += gridDim.x * nw) {
            const R* col = Ainv + cp.moff + (long long)row * cp.n0;  // symmetric: column = row
            R s = R(0);
            if (sizeof(R) == 4 && (cp.n0 & 3) == 0 && (cp.moff & 3) == 0) {
                // 16-byte loads, four partial sums per lane (fixed order)
                const float4* c4 = reinterpret_cast<const float4*>(col);
                const float4* g4 = reinterpret_cast<const float4*>(gs);
                float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 8
                for (int j = lane; j < (cp.n0 >> 2); j += 32) {
                    const float4 m = __ldg(c4 + j), q = g4[j];
                    a0 += m.x * q.x; a1 += m.y * q.y; a2 += m.z * q.z; a3 += m.w * q.w;
                }
                s = (R)((a0 + a1) + (a2 + a3));
            } else {
                for (int j = lane; j < cp.n0; j += 32) s += col[j] * gs[j];
            }
            s = warp_sum(s);
            if (lane == 0) {
                yv[cp.voff + row] = s;
                P.gy[cp.voff + row] = (double)s * (double)gs[row];
            }
        }
        __syncthreads();
    }
    if (P.apply_only) return;
    if (!arrive_last(P.counter, gridDim.x, &sh_last)) return;
    for (int pi = 0; pi < P.npairs; ++pi) {
        PairScalars* sp = P.sc + pi;
        if (sp->done) continue;
        const PairDesc pd = P.pairs[pi];
        const CoarsePair cp = P.cps[pi];
        const int ntp = pd.tiles_x * pd.tiles_y;
        const double t_rr = ordered_sum_rt(P.tpart + 2 * (long long)pd.tile0, ntp, 2, sh_red);
        const double t_rz = ordered_sum_rt(P.tpart + 2 * (long long)pd.tile0 + 1, ntp, 2, sh_red);
        const double t_gy = ordered_sum_rt(P.gy + cp.voff, cp.n0, 1, sh_red);
        if (threadIdx.x == 0) precond_finalize(sp, t_rr, t_rz + t_gy, P.first);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (P.use_cond) {
            int more = 0;
            for (int pi = 0; pi < P.npairs; ++pi) more |= !P.sc[pi].done;
            if (*(volatile int*)P.err) more = 0;
            cudaGraphSetConditional(P.cond, more ? 1u : 0u);
        }
        __threadfence();
        *P.counter = 0u;
    }
}

// z += R_0^T y: bilinear interpolation of the coarse correction, one warp
// per row, lanes along x
template <typename R>
__global__ void __launch_bounds__(256) k_coarse_prolong(const PairDesc* pairs, const CoarsePair* cps,
                                                        const CoarseCell* cells, const PairScalars* sc,
                                                        int skip_done, int only_pair, const R* __restrict__ yv,
                                                        R* __restrict__ za) {
    const CoarseCell c = cells[blockIdx.x];
    if ((skip_done && sc[c.pair].done) || (only_pair >= 0 && c.pair != only_pair)) return;
    const PairDesc pd = pairs[c.pair];
    const CoarsePair cp = cps[c.pair];
    const long long plane = (long long)pd.H * pd.pitch;
    R yc[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int k = c.k + (a & 1), l = c.l + (a >> 1);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) yc[a][cc] = yv[cp.voff + 3 * ((long long)l * cp.nx + k) + cc];
    }
    int nx, ny;
    cell_nodes(c, cp, nx, ny);
    const R ix = R(1) / R(c.x1 - c.x0), iy = R(1) / R(c.y1 - c.y0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int yy = warp; yy < ny; yy += nw) {
        R* row = za + pd.vec_off + (long long)(c.y0 + yy) * pd.pitch + c.x0;
        const R wy = R(yy) * iy;
        R e0[3], e1[3];  // the coarse correction at the row's two cell edges
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            e0[cc] = (R(1) - wy) * yc[0][cc] + wy * yc[2][cc];
            e1[cc] = (R(1) - wy) * yc[1][cc] + wy * yc[3][cc];
        }
        for (int x0 = 0; x0 < nx; x0 += 128) {
            R zv[4][3];
#pragma unroll
            for (int u = 0; u < 4; ++u) {  // loads of the row before its stores
                const int xx = x0 + lane + 32 * u;
                if (xx < nx) { zv[u][0] = row[xx]; zv[u][1] = row[xx + plane]; zv[u][2] = row[xx + 2 * plane]; }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int xx = x0 + lane + 32 * u;
                if (xx >= nx) continue;
                const R wx = R(xx) * ix;
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    row[xx + cc * plane] = zv[u][cc] + ((R(1) - wx) * e0[cc] + wx * e1[cc]);
            }
        }
    }
}

// ----------------------------------------------------------- launchers --
cudaError_t launch_coarse_assemble(const SolveBufs& B, cudaStream_t st) {
    const CoarseBufs& C = B.coarse;
    if (B.fp64)
        k_coarse_assemble<double><<<C.ncells, 256, 0, st>>>(B.pairs, C.cps, C.cells, (const double*)B.f1,
                                                            (const double*)B.f2, (const double*)B.alpha, B.lam, B.gms,
                                                            (double*)C.blk);
    else
        k_coarse_assemble<float><<<C.ncells, 256, 0, st>>>(B.pairs, C.cps, C.cells, (const float*)B.f1,
                                                           (const float*)B.f2, (const float*)B.alpha, B.lam, B.gms,
                                                           (float*)C.blk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long items = C.scatter_items;
    const unsigned g = (unsigned)((items + 255) / 256);
    if (B.fp64) k_coarse_scatter<double><<<g, 256, 0, st>>>(C.cps, B.npairs, (const double*)C.blk, (double*)C.Amat);
    else k_coarse_scatter<float><<<g, 256, 0, st>>>(C.cps, B.npairs, (const float*)C.blk, (float*)C.Amat);
    return cudaGetLastError();
}

cudaError_t launch_symmetrize(void* A, int fp64, int n, cudaStream_t st);

cudaError_t launch_coarse_factor(const SolveBufs& B, int pair, int n0, int nx, long long moff, cudaStream_t st) {
    const CoarseBufs& C = B.coarse;
    const int b = 3 * nx + 5, w = b + 1;
    const size_t es = B.fp64 ? 8 : 4;
    const size_t smem_c = ((size_t)w * w + w) * es, smem_i = (size_t)inv_smem_elems(b) * es;
    const size_t smem_b = (size_t)cb_smem_elems(b) * es;
    if (smem_b <= kMaxSmem) {
        const int nt = cb_threads(b);
        const unsigned gr = (unsigned)(((long long)n0 * w + 255) / 256);
        if (B.fp64) {
            k_band_cholesky_blk<double><<<1, nt, smem_b, st>>>(C.cps, pair, b, (const double*)C.Amat,
                                                                (double*)C.Lc, C.info);
            k_band_rows<double><<<gr, 256, 0, st>>>(C.cps, pair, b, (const double*)C.Lc, (double*)C.Lr);
        } else {
            k_band_cholesky_blk<float><<<1, nt, smem_b, st>>>(C.cps, pair, b, (const float*)C.Amat, (float*)C.Lc,
                                                               C.info);
            k_band_rows<float><<<gr, 256, 0, st>>>(C.cps, pair, b, (const float*)C.Lc, (float*)C.Lr);
        }
    } else if (B.fp64)
        k_band_cholesky<double><<<1, 1024, smem_c, st>>>(C.cps, pair, b, (const double*)C.Amat, (double*)C.Lr,
                                                         (double*)C.Lc, C.info);
    else
        k_band_cholesky<float><<<1, 1024, smem_c, st>>>(C.cps, pair, b, (const float*)C.Amat, (float*)C.Lr,
                                                        (float*)C.Lc, C.info);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)((n0 + INV_WARPS - 1) / INV_WARPS);
    if (B.fp64)
        k_band_inverse<double><<<g, INV_WARPS * 32, smem_i, st>>>(C.cps, pair, b, (const double*)C.Lr, (const double*)C.Lc,
                                                       (double*)C.Ainv);
    else
        k_band_inverse<float><<<g, INV_WARPS * 32, smem_i, st>>>(C.cps, pair, b, (const float*)C.Lr, (const float*)C.Lc,
                                                      (float*)C.Ainv);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_symmetrize((char*)C.Ainv + (size_t)moff * es, B.fp64, n0, st);
}

cudaError_t launch_symmetrize(void* A, int fp64, int n, cudaStream_t st) {
    const dim3 b(32, 8), g((n + 31) / 32, (n + 7) / 8);
    if (fp64) k_symmetrize<double><<<g, b, 0, st>>>((double*)A, n);
    else k_symmetrize<float><<<g, b, 0, st>>>((float*)A, n);
    return cudaGetLastError();
}

cudaError_t launch_coarse_apply(const SolveBufs& B, int first, int apply_only, int use_cond,
                                cudaGraphConditionalHandle cond, int only_pair, cudaStream_t st) {
    const CoarseBufs& C = B.coarse;
    const int skip = apply_only ? 0 : 1;
    if (B.fp64)
        k_coarse_restrict<double><<<C.ncells, 256, 0, st>>>(B.pairs, C.cps, C.cells, B.sc, skip, only_pair,
                                                            (const double*)B.r, (double*)C.part);
    else
        k_coarse_restrict<float><<<C.ncells, 256, 0, st>>>(B.pairs, C.cps, C.cells, B.sc, skip, only_pair,
                                                           (const float*)B.r, (float*)C.part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CoarseParams P;
    memset(&P, 0, sizeof(P));
    P.pairs = B.pairs;
    P.cps = C.cps;
    P.npairs = B.npairs;
    P.sc = B.sc;
    P.tpart = B.partS;
    P.Ainv = C.Ainv;
    P.part = C.part;
    P.y = C.y;
    P.gy = C.gy;
    P.counter = C.cnt;
    P.err = B.err;
    P.first = first;
    P.apply_only = apply_only;
    P.use_cond = use_cond;
    P.cond = cond;
    P.only_pair = only_pair;
    P.g = C.g;
    const int total = C.total_n0;
    if (B.fp64) k_coarse_gather_d<<<(total + 255) / 256, 256, 0, st>>>(P, total);
    else k_coarse_gather_f<<<(total + 255) / 256, 256, 0, st>>>(P, total);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)C.max_n0 * (B.fp64 ? 8 : 4);
    if (B.fp64) k_coarse_gemv<double><<<C.gemv_grid, 256, smem, st>>>(P);
    else k_coarse_gemv<float><<<C.gemv_grid, 256, smem, st>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (B.fp64)
        k_coarse_prolong<double><<<C.ncells, 256, 0, st>>>(B.pairs, C.cps, C.cells, B.sc, skip, only_pair,
                                                           (const double*)C.y, (double*)B.z);
    else
        k_coarse_prolong<float><<<C.ncells, 256, 0, st>>>(B.pairs, C.cps, C.cells, B.sc, skip, only_pair,
                                                          (const float*)C.y, (float*)B.z);
    return cudaGetLastError();
}

cudaError_t coarse_configure(int fp64, int max_n0, int max_nx) {
    const size_t es = fp64 ? 8 : 4;
    const int w = 3 * max_nx + 6;
    const int s_gemv = (int)(max_n0 * es), s_chol = (int)(((size_t)w * w + w) * es), s_inv = (int)(inv_smem_elems(w - 1) * es);
    cudaError_t e = cudaSuccess;
    const size_t s_blk = (size_t)cb_smem_elems(w - 1) * es;
    if (s_blk <= kMaxSmem) {
        e = fp64 ? cudaFuncSetAttribute(k_band_cholesky_blk<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_blk)
                 : cudaFuncSetAttribute(k_band_cholesky_blk<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_blk);
        if (e != cudaSuccess) return e;
    }
    if (fp64) {
        e = cudaFuncSetAttribute(k_coarse_gemv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, s_gemv);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_band_cholesky<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, s_chol);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_band_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, s_inv);
    } else {
        e = cudaFuncSetAttribute(k_coarse_gemv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, s_gemv);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_band_cholesky<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, s_chol);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_band_inverse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, s_inv);
    }
    return e;
}

}  // namespace ofl
