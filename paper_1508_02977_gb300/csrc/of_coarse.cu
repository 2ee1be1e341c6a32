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

#include "of_common.cuh"
#include "of_launch.h"
#include "of_schwarz.cuh"

namespace ofl {

using namespace ofk;

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
    // thread map of the trailing update: 8 threads per row offset a, columns c = 1 + t8 + 8 q
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
        // slot sj now takes row j + w: columns j+1 .. j+w
        if ((int)threadIdx.x < w) {
            int rc = sj + 1 + (int)threadIdx.x;
            if (rc >= w) rc -= w;
            Wn[sj * w + rc] = cur;
        }
        __syncthreads();
        if (++sj == w) sj = 0;
    }
    if (threadIdx.x == 0 && !bad) info[pair] = 0;
}

// Dense inverse X = A_0^{-1} = L^{-T} L^{-1}, one warp per column i:
// forward L y = e_i (y_k = 0 for k < i), backward L^T x = y.  The last b+1
// values of the running solution stay in a per-warp ring in shared memory;
// each lane holds up to NPL factor entries of a row, and the next row's are
// loaded while the current one is reduced.
template <typename R>
__global__ void __launch_bounds__(256) k_band_inverse(const CoarsePair* cps, int pair, int b,
                                                      const R* __restrict__ Lr, const R* __restrict__ Lc,
                                                      R* __restrict__ X) {
    constexpr int NPL = 8;  // b + 1 <= 32 NPL
    extern __shared__ __align__(16) unsigned char rsm[];
    const int w = b + 1, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    R* ring = reinterpret_cast<R*>(rsm) + (size_t)warp * w;
    const CoarsePair cp = cps[pair];
    const int n = cp.n0;
    const int i = blockIdx.x * (blockDim.x >> 5) + warp;
    if (i >= n) return;
    const R* Lrp = Lr + cp.boff;
    const R* Lcp = Lc + cp.boff;
    R* xcol = X + cp.moff + (long long)i * n;
    for (int t = lane; t < w; t += 32) ring[t] = R(0);
    __syncwarp();
    // forward, row r: entries L[r][r-o], o = 1..min(b, r-i) (offset o by lane l + 32 q)
    R cur[NPL], nxt[NPL];
    auto load_f = [&](int r, R (&dst)[NPL]) {
#pragma unroll
        for (int q = 0; q < NPL; ++q) {
            const int o = 1 + lane + 32 * q;
            dst[q] = (r < n && o <= b && o <= r - i) ? Lrp[(long long)r * w + o] : R(0);
        }
    };
    load_f(i, cur);
    R diag = Lrp[(long long)i * w];
    int rm = i % w;  // r mod w
    for (int r = i; r < n; ++r) {
        const R dnext = (r + 1 < n) ? Lrp[(long long)(r + 1) * w] : R(1);
        load_f(r + 1, nxt);
        R s = R(0);
#pragma unroll
        for (int q = 0; q < NPL; ++q) {
            const int o = 1 + lane + 32 * q;
            if (o <= b && o <= r - i) {
                int sl = rm - o;
                if (sl < 0) sl += w;
                s += cur[q] * ring[sl];
            }
        }
        s = warp_sum(s);
        const R yr = ((r == i ? R(1) : R(0)) - s) / diag;
        __syncwarp();
        if (lane == 0) { ring[rm] = yr; xcol[r] = yr; }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NPL; ++q) cur[q] = nxt[q];
        diag = dnext;
        if (++rm == w) rm = 0;
    }
    for (int t = lane; t < i; t += 32) xcol[t] = R(0);
    for (int t = lane; t < w; t += 32) ring[t] = R(0);
    __syncwarp();
    // backward, row r: entries L[r+o][r], o = 1..min(b, n-1-r)
    auto load_b = [&](int r, R (&dst)[NPL]) {
#pragma unroll
        for (int q = 0; q < NPL; ++q) {
            const int o = 1 + lane + 32 * q;
            dst[q] = (r >= 0 && o <= b && r + o < n) ? Lcp[(long long)r * w + o] : R(0);
        }
    };
    load_b(n - 1, cur);
    diag = Lcp[(long long)(n - 1) * w];
    rm = (n - 1) % w;
    for (int r = n - 1; r >= 0; --r) {
        const R dnext = (r > 0) ? Lcp[(long long)(r - 1) * w] : R(1);
        load_b(r - 1, nxt);
        R s = R(0);
#pragma unroll
        for (int q = 0; q < NPL; ++q) {
            const int o = 1 + lane + 32 * q;
            if (o <= b && r + o < n) {
                int sl = rm + o;
                if (sl >= w) sl -= w;
                s += cur[q] * ring[sl];
            }
        }
        s = warp_sum(s);
        const R xr = (xcol[r] - s) / diag;
        __syncwarp();
        if (lane == 0) { ring[rm] = xr; xcol[r] = xr; }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NPL; ++q) cur[q] = nxt[q];
        diag = dnext;
        if (--rm < 0) rm = w - 1;
    }
}

// ---------------------------------------------------------- application --
// g-partials of a cell: sum over its nodes of hat_a(node) r_c(node)
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
    const R* r = ra + pd.vec_off;
    int nx, ny;
    cell_nodes(c, cp, nx, ny);
    R acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = R(0);
    const int nn = nx * ny, step = blockDim.x;
    for (int i0 = threadIdx.x; i0 < nn; i0 += 4 * step) {
        R v[4][3];
        long long oo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {  // loads of four nodes first
            const int i = i0 + u * step;
            oo[u] = -1;
            if (i < nn) {
                const int x = c.x0 + i % nx, y = c.y0 + i / nx;
                oo[u] = (long long)y * pd.pitch + x;
                v[u][0] = r[oo[u]];
                v[u][1] = r[oo[u] + plane];
                v[u][2] = r[oo[u] + 2 * plane];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * step;
            if (i >= nn) continue;
            R ph[4];
            cell_hats<R>(c.x0 + i % nx, c.y0 + i / nx, c, ph);
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) acc[3 * a + cc] += ph[a] * v[u][cc];
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
        for (int u = threadIdx.x; u < cp.n0; u += blockDim.x) gs[u] = gg[u];
        __syncthreads();
        for (int row = blockIdx.x * nw + warp; row < cp.n0; row += gridDim.x * nw) {
            const R* col = Ainv + cp.moff + (long long)row * cp.n0;  // symmetric: column = row
            R s = R(0);
            for (int j = lane; j < cp.n0; j += 32) s += col[j] * gs[j];
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

// z += R_0^T y: bilinear interpolation of the coarse correction
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
    R* z = za + pd.vec_off;
    R yc[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int k = c.k + (a & 1), l = c.l + (a >> 1);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) yc[a][cc] = yv[cp.voff + 3 * ((long long)l * cp.nx + k) + cc];
    }
    int nx, ny;
    cell_nodes(c, cp, nx, ny);
    const int nn = nx * ny, step = blockDim.x;
    for (int i0 = threadIdx.x; i0 < nn; i0 += 4 * step) {
        R zv[4][3];
        long long oo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {  // loads of four nodes first
            const int i = i0 + u * step;
            oo[u] = -1;
            if (i < nn) {
                oo[u] = (long long)(c.y0 + i / nx) * pd.pitch + (c.x0 + i % nx);
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) zv[u][cc] = z[oo[u] + cc * plane];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * step;
            if (i >= nn) continue;
            R ph[4];
            cell_hats<R>(c.x0 + i % nx, c.y0 + i / nx, c, ph);
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
                z[oo[u] + cc * plane] =
                    zv[u][cc] + (ph[0] * yc[0][cc] + ph[1] * yc[1][cc] + ph[2] * yc[2][cc] + ph[3] * yc[3][cc]);
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
    const size_t smem_c = ((size_t)w * w + w) * es, smem_i = (size_t)8 * w * es;
    if (B.fp64)
        k_band_cholesky<double><<<1, 1024, smem_c, st>>>(C.cps, pair, b, (const double*)C.Amat, (double*)C.Lr,
                                                         (double*)C.Lc, C.info);
    else
        k_band_cholesky<float><<<1, 1024, smem_c, st>>>(C.cps, pair, b, (const float*)C.Amat, (float*)C.Lr,
                                                        (float*)C.Lc, C.info);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)((n0 + 7) / 8);
    if (B.fp64)
        k_band_inverse<double><<<g, 256, smem_i, st>>>(C.cps, pair, b, (const double*)C.Lr, (const double*)C.Lc,
                                                       (double*)C.Ainv);
    else
        k_band_inverse<float><<<g, 256, smem_i, st>>>(C.cps, pair, b, (const float*)C.Lr, (const float*)C.Lc,
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
    const int s_gemv = (int)(max_n0 * es), s_chol = (int)(((size_t)w * w + w) * es), s_inv = (int)(8 * w * es);
    cudaError_t e = cudaSuccess;
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
