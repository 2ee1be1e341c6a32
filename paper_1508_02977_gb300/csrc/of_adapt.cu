// Error indicator and alpha update (Section 2.3, Eq. errind and the update
// formula that follows it), and the adjoint gradients of a loss through the
// solve (implicit differentiation of A(theta) U = b(theta)).
#include <cuda_runtime.h>

#include "of_common.cuh"
#include "of_launch.h"

namespace ofl {

using namespace ofk;

// U (3 components) at node (x, y) of the solution planes (FP64, or an FP32
// copy on the FP32 path), as R.
template <typename R, typename UT>
struct UView {
    const UT* u;
    long long plane;
    int pitch;
    __device__ __forceinline__ void at(int x, int y, R v[3]) const {
        const long long o = (long long)y * pitch + x;
        v[0] = (R)u[o];
        v[1] = (R)u[o + plane];
        v[2] = (R)u[o + 2 * plane];
    }
};

// gradient of the P1 interpolant of U on triangle t of square (X,Y) from the
// corner values A=(X,Y) B=(X+1,Y) C=(X+1,Y+1) D=(X,Y+1)
template <typename R>
__device__ __forceinline__ void tri_grad(int t, const R A[3], const R B[3], const R C[3], const R D[3], R gx[3],
                                         R gy[3]) {
    for (int c = 0; c < 3; ++c) {
        if (t == 0) { gx[c] = B[c] - A[c]; gy[c] = C[c] - B[c]; }
        else        { gx[c] = C[c] - D[c]; gy[c] = D[c] - A[c]; }
    }
}

// ------------------------------------------------------------ indicator --
// One thread per square; eta of both triangles.
//   interior: h_K || Lambda^{-1/2} R ||_{L2(K)},  R = -g (g.U_h + ft), by the
//             edge-midpoint rule (exact here): (|K|/3) G sum_m s_m^2,
//             G = sum_c g_c^2 / Lambda_c, s_m = ft + g.U_h(midpoint m);
//   edges:    (1/2) h_e |Lambda_e^{-1/2} J_e|  (J_e constant on the edge, so
//             h_e^{1/2} ||.||_{L2(e)} = h_e |.|), J_e = outside - inside flux,
//             outside flux 0 on the image boundary, Lambda_e = max of the two.
template <typename R, typename UT>
__global__ void k_indicator(const PairDesc* pairs, int pair, const R* __restrict__ f1a, const R* __restrict__ f2a,
                            const R* __restrict__ ala, const UT* __restrict__ ua, R* __restrict__ etaa, R lam, R gms,
                            const R* __restrict__ eld, long long eld_stride, const R* __restrict__ lama,
                            unsigned long long* __restrict__ etamax_bits) {
    const PairDesc pd = pairs[pair];
    const int W = pd.W, H = pd.H, pitch = pd.pitch;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    // the running max in the storage type (max is exact; one conversion per
    // warp: FP64 instructions per element would run on the narrow FP64 pipe)
    R lmax = R(0);
    if (x < W - 1 && y < H - 1) {
        const R* f1 = f1a + pd.frame_off;
        const R* f2 = f2a + pd.frame_off;
        const R* al = ala + 2 * pd.frame_off;
        UView<R, UT> U{ua + pd.vec_off, (long long)H * pitch, pitch};
        const R ilam = R(1) / lam;  // Lambda^{-1} enters as products with reciprocals; gms: of_model scale
        auto F1 = [&](int xx, int yy) { return f1[(long long)yy * pitch + xx]; };
        auto F2 = [&](int xx, int yy) { return f2[(long long)yy * pitch + xx]; };
        auto AL = [&](int xx, int yy, int t) { return al[2 * ((long long)yy * pitch + xx) + t]; };
        // lambda of an element: the per-element field when given, else the constant
        const R* la = lama ? lama + 2 * pd.frame_off : nullptr;
        auto LA = [&](int xx, int yy, int t) { return la ? la[2 * ((long long)yy * pitch + xx) + t] : lam; };
        R uA[3], uB[3], uC[3], uD[3];
        U.at(x, y, uA); U.at(x + 1, y, uB); U.at(x + 1, y + 1, uC); U.at(x, y + 1, uD);
        R gxK[2][3], gyK[2][3];
        tri_grad<R>(0, uA, uB, uC, uD, gxK[0], gyK[0]);
        tri_grad<R>(1, uA, uB, uC, uD, gxK[1], gyK[1]);
        const R aK[2] = {AL(x, y, 0), AL(x, y, 1)};
        const R third = R(1) / R(3);
        const R sq2 = R(1.4142135623730951);
        R* eta = etaa + 2 * pd.frame_off;
        for (int t = 0; t < 2; ++t) {
            // element data
            const R* V1 = (t == 0) ? uB : uD;  // middle vertex
            R g0, g1, g2, ft;
            if (t == 0) {
                g0 = F2(x + 1, y) - F2(x, y); g1 = F2(x + 1, y + 1) - F2(x + 1, y);
                g2 = -(F1(x, y) + F1(x + 1, y) + F1(x + 1, y + 1)) * third * gms;
                ft = ((F2(x, y) - F1(x, y)) + (F2(x + 1, y) - F1(x + 1, y)) + (F2(x + 1, y + 1) - F1(x + 1, y + 1))) * third;
            } else {
                g0 = F2(x + 1, y + 1) - F2(x, y + 1); g1 = F2(x, y + 1) - F2(x, y);
                g2 = -(F1(x, y) + F1(x, y + 1) + F1(x + 1, y + 1)) * third * gms;
                ft = ((F2(x, y) - F1(x, y)) + (F2(x, y + 1) - F1(x, y + 1)) + (F2(x + 1, y + 1) - F1(x + 1, y + 1))) * third;
            }
            const R lK = la ? LA(x, y, t) : lam, ilK = la ? R(1) / lK : ilam;
            const R Lk[3] = {aK[t], aK[t], lK};
            const R iaK = R(1) / aK[t];
            const R iLk[3] = {iaK, iaK, ilK};
            const R G = (g0 * g0 + g1 * g1) * iaK + g2 * g2 * ilK;
            // midpoints of the 3 edges: (A,V1), (V1,C), (C,A)
            R sm2 = R(0);
            const R* P0[3] = {uA, V1, uC};
            R val;
            if (!eld) {  // R = F - A U = -g (g.U + ft)
                for (int e = 0; e < 3; ++e) {
                    const R* Pa = P0[e];
                    const R* Pb = P0[(e + 1) % 3];
                    const R s = ft + R(0.5) * (g0 * (Pa[0] + Pb[0]) + g1 * (Pa[1] + Pb[1]) + g2 * (Pa[2] + Pb[2]));
                    sm2 += s * s;
                }
                val = sq2 * sqrt(R(0.5) / R(3) * G * sm2);
            } else {     // K_rho element data: R = F - A_rho U
                const R* ep = eld + pd.frame_off + (long long)y * pitch + x + (long long)(9 * t) * eld_stride;
                R a[6], fv[3];
                for (int k = 0; k < 6; ++k) a[k] = ep[k * eld_stride];
                for (int k = 0; k < 3; ++k) fv[k] = ep[(6 + k) * eld_stride];
                for (int e = 0; e < 3; ++e) {
                    const R* Pa = P0[e];
                    const R* Pb = P0[(e + 1) % 3];
                    const R m0 = R(0.5) * (Pa[0] + Pb[0]), m1 = R(0.5) * (Pa[1] + Pb[1]), m2 = R(0.5) * (Pa[2] + Pb[2]);
                    const R r0 = fv[0] - (a[0] * m0 + a[1] * m1 + a[2] * m2);
                    const R r1 = fv[1] - (a[1] * m0 + a[3] * m1 + a[4] * m2);
                    const R r2 = fv[2] - (a[2] * m0 + a[4] * m1 + a[5] * m2);
                    sm2 += (r0 * r0 + r1 * r1) * iLk[0] + r2 * r2 * iLk[2];
                }
                val = sq2 * sqrt(R(0.5) / R(3) * sm2);
            }
            // edges: normal, length, neighbour (square, t) or none
            for (int e = 0; e < 3; ++e) {
                R nx, ny, he;
                int nbx = 0, nby = 0, nbt = 0;
                bool has = false;
                if (t == 0) {
                    if (e == 0) { nx = 0; ny = -1; he = 1; has = y >= 1; nbx = x; nby = y - 1; nbt = 1; }
                    else if (e == 1) { nx = 1; ny = 0; he = 1; has = x + 1 <= W - 2; nbx = x + 1; nby = y; nbt = 1; }
                    else { nx = -R(0.7071067811865476); ny = R(0.7071067811865476); he = sq2; has = true; nbx = x; nby = y; nbt = 1; }
                } else {
                    if (e == 0) { nx = -1; ny = 0; he = 1; has = x >= 1; nbx = x - 1; nby = y; nbt = 0; }
                    else if (e == 1) { nx = 0; ny = 1; he = 1; has = y + 1 <= H - 2; nbx = x; nby = y + 1; nbt = 0; }
                    else { nx = R(0.7071067811865476); ny = -R(0.7071067811865476); he = sq2; has = true; nbx = x; nby = y; nbt = 0; }
                }
                R ngx[3] = {0, 0, 0}, ngy[3] = {0, 0, 0};
                R aO = R(0), iaO = R(0), lO = lam, ilO = ilam;
                if (has) {
                    R qA[3], qB[3], qC[3], qD[3];
                    if (nbx == x && nby == y) {
                        for (int c = 0; c < 3; ++c) { ngx[c] = gxK[nbt][c]; ngy[c] = gyK[nbt][c]; }
                    } else {
                        U.at(nbx, nby, qA); U.at(nbx + 1, nby, qB); U.at(nbx + 1, nby + 1, qC); U.at(nbx, nby + 1, qD);
                        tri_grad<R>(nbt, qA, qB, qC, qD, ngx, ngy);
                    }
                    aO = AL(nbx, nby, nbt);
                    iaO = R(1) / aO;
                    if (la) {
                        lO = LA(nbx, nby, nbt);
                        ilO = R(1) / lO;
                    }
                }
                R q = R(0);
                for (int c = 0; c < 3; ++c) {
                    const R lk = Lk[c];
                    const R lo = (c < 2) ? aO : lO;
                    const R fin = lk * (gxK[t][c] * nx + gyK[t][c] * ny);
                    const R fout = has ? lo * (ngx[c] * nx + ngy[c] * ny) : R(0);
                    // 1 / max(lo, lk) = min(1/lo, 1/lk)
                    const R ilo = (c < 2) ? iaO : ilO;
                    const R ile = has ? (ilo < iLk[c] ? ilo : iLk[c]) : iLk[c];
                    const R J = fout - fin;
                    q += J * J * ile;
                }
                val += R(0.5) * he * sqrt(q);
            }
            eta[2 * ((long long)y * pitch + x) + t] = val;
            lmax = val > lmax ? val : lmax;
        }
    }
    lmax = warp_max(lmax);
    if ((threadIdx.x & 31) == 0 && lmax > R(0))
        atomicMax(etamax_bits + pair, (unsigned long long)__double_as_longlong((double)lmax));
}

// kappa, eta_thr, alpha_th come in the storage type; 1 / max(eta) is formed
// (in FP64, then rounded) once per block rather than per thread.
template <typename R>
__global__ void k_alpha_update(const PairDesc* pairs, int pair, R* __restrict__ ala, const R* __restrict__ etaa,
                               const unsigned long long* __restrict__ etamax_bits, R kappa, R eta_thr, R alpha_th) {
    __shared__ R s_im;
    __shared__ int s_on;
    const PairDesc pd = pairs[pair];
    const int W = pd.W, pitch = pd.pitch;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (threadIdx.x == 0) {
        const double m = __longlong_as_double((long long)etamax_bits[pair]);
        s_on = m > 0.0;
        s_im = s_on ? (R)(1.0 / m) : R(0);
    }
    __syncthreads();
    if (x >= W - 1 || !s_on) return;
    R* al = ala + 2 * pd.frame_off;
    const R* eta = etaa + 2 * pd.frame_off;
    const R im = s_im;
    for (int t = 0; t < 2; ++t) {
        const long long o = 2 * ((long long)y * pitch + x) + t;
        const R rel = eta[o] * im - eta_thr;
        const R a = al[o] / (R(1) + kappa * (rel > R(0) ? rel : R(0)));
        al[o] = a > alpha_th ? a : alpha_th;
    }
}

cudaError_t launch_indicator(const AdaptBufs& A, int pair, int H, int W, cudaStream_t st) {
    dim3 grid((W - 1 + 127) / 128, H - 1);
    if (A.fp64)
        k_indicator<double, double><<<grid, 128, 0, st>>>(A.pairs, pair, (const double*)A.f1, (const double*)A.f2,
                                                          (const double*)A.alpha, A.u, (double*)A.eta, A.lam, A.gms,
                                                          (const double*)A.eld, A.eld_stride, (const double*)A.lamel,
                                                          (unsigned long long*)A.etamax);
    else
        k_indicator<float, float><<<grid, 128, 0, st>>>(A.pairs, pair, (const float*)A.f1, (const float*)A.f2,
                                                        (const float*)A.alpha, A.u32, (float*)A.eta, (float)A.lam,
                                                        (float)A.gms,
                                                        (const float*)A.eld, A.eld_stride, (const float*)A.lamel,
                                                        (unsigned long long*)A.etamax);
    return cudaGetLastError();
}

cudaError_t launch_alpha_update(const AdaptBufs& A, int pair, int H, int W, double kappa, double eta_thr,
                                double alpha_th, cudaStream_t st, void* field) {
    // field: the per-element parameter updated by the rule (alpha, or the
    // per-element lambda with its own threshold)
    void* f = field ? field : A.alpha;
    dim3 grid((W - 1 + 127) / 128, H - 1);
    if (A.fp64)
        k_alpha_update<double><<<grid, 128, 0, st>>>(A.pairs, pair, (double*)f, (const double*)A.eta,
                                                     (const unsigned long long*)A.etamax, kappa, eta_thr, alpha_th);
    else
        k_alpha_update<float><<<grid, 128, 0, st>>>(A.pairs, pair, (float*)f, (const float*)A.eta,
                                                    (const unsigned long long*)A.etamax, (float)kappa, (float)eta_thr,
                                                    (float)alpha_th);
    return cudaGetLastError();
}

// -------------------------------------------------------------- adjoint --
// Per element, with s_i = g.U_i, t_i = g.Lam_i (vertex i), the adjoint-weighted
// element residual is
//   E_K = |K|/12 sum_ij (1+d_ij) t_i s_j + |K|/3 ft sum_i t_i
//         + |K| sum_c Lambda_c grad Lam_c . grad U_c
// and dL/dtheta = -dE_K/dtheta.  Through g and ft:
//   dE/dg_c = |K|/12 [sum_i (Lam_ic s_i + t_i U_ic) + (sum_i Lam_ic)(sum s)
//             + (sum t)(sum_i U_ic)] + |K|/3 ft sum_i Lam_ic,
//   dE/dft  = |K|/3 sum t.
template <typename R>
__device__ __forceinline__ void elem_adjoint(const R u[3][3], const R l[3][3], const R g[3], R ft, R dEdg[3], R& dEdft) {
    R s[3], tt[3];
    for (int i = 0; i < 3; ++i) {
        s[i] = g[0] * u[i][0] + g[1] * u[i][1] + g[2] * u[i][2];
        tt[i] = g[0] * l[i][0] + g[1] * l[i][1] + g[2] * l[i][2];
    }
    const R Ss = s[0] + s[1] + s[2], St = tt[0] + tt[1] + tt[2];
    const R k12 = R(0.5) / R(12), k3 = R(0.5) / R(3);
    for (int c = 0; c < 3; ++c) {
        R a = R(0), Lc = R(0), Uc = R(0);
        for (int i = 0; i < 3; ++i) {
            a += l[i][c] * s[i] + tt[i] * u[i][c];
            Lc += l[i][c];
            Uc += u[i][c];
        }
        dEdg[c] = k12 * (a + Lc * Ss + St * Uc) + k3 * ft * Lc;
    }
    dEdft = k3 * St;
}

// dL/dalpha: one thread per square, both triangles.
template <typename R, typename O>
__global__ void k_adjoint_alpha(const PairDesc* pairs, int pair, const double* __restrict__ ua,
                                const double* __restrict__ la, O* __restrict__ out) {
    const PairDesc pd = pairs[pair];
    const int W = pd.W, H = pd.H, pitch = pd.pitch;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W - 1 || y >= H - 1) return;
    UView<R, double> U{ua + pd.vec_off, (long long)H * pitch, pitch};
    UView<R, double> L{la + pd.vec_off, (long long)H * pitch, pitch};
    R uA[3], uB[3], uC[3], uD[3], lA[3], lB[3], lC[3], lD[3];
    U.at(x, y, uA); U.at(x + 1, y, uB); U.at(x + 1, y + 1, uC); U.at(x, y + 1, uD);
    L.at(x, y, lA); L.at(x + 1, y, lB); L.at(x + 1, y + 1, lC); L.at(x, y + 1, lD);
    for (int t = 0; t < 2; ++t) {
        R ugx[3], ugy[3], lgx[3], lgy[3];
        tri_grad<R>(t, uA, uB, uC, uD, ugx, ugy);
        tri_grad<R>(t, lA, lB, lC, lD, lgx, lgy);
        R s = R(0);
        for (int c = 0; c < 2; ++c) s += lgx[c] * ugx[c] + lgy[c] * ugy[c];
        out[((long long)y * (W - 1) + x) * 2 + t] = (O)(-R(0.5) * s);
    }
}

// dL/df2 and dL/df1: one thread per node, gathering its 6 elements
//   E1 = sq(x,y).t0 (node is a), E2 = sq(x,y).t1 (a), E3 = sq(x-1,y-1).t0 (c),
//   E4 = sq(x-1,y-1).t1 (c), E5 = sq(x-1,y).t0 (b), E6 = sq(x,y-1).t1 (d),
// with the node's basis gradient in each: (-1,0) (0,-1) (0,1) (1,0) (1,-1) (-1,1).
template <typename R, typename O>
__global__ void k_adjoint_frames(const PairDesc* pairs, int pair, const R* __restrict__ f1a, const R* __restrict__ f2a,
                                 const double* __restrict__ ua, const double* __restrict__ la, O* __restrict__ df2,
                                 O* __restrict__ df1, double gms_d) {
    const PairDesc pd = pairs[pair];
    const R gms = (R)gms_d;
    const int W = pd.W, H = pd.H, pitch = pd.pitch;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const R* f1 = f1a + pd.frame_off;
    const R* f2 = f2a + pd.frame_off;
    UView<R, double> U{ua + pd.vec_off, (long long)H * pitch, pitch};
    UView<R, double> L{la + pd.vec_off, (long long)H * pitch, pitch};
    const int sqx[6] = {x, x, x - 1, x - 1, x - 1, x};
    const int sqy[6] = {y, y, y - 1, y - 1, y, y - 1};
    const int sqt[6] = {0, 1, 0, 1, 0, 1};
    const R phx[6] = {-1, 0, 0, 1, 1, -1};
    const R phy[6] = {0, -1, 1, 0, -1, 1};
    const R third = R(1) / R(3);
    R a2 = R(0), a1 = R(0);
    for (int e = 0; e < 6; ++e) {
        const int X = sqx[e], Y = sqy[e], t = sqt[e];
        if (X < 0 || Y < 0 || X >= W - 1 || Y >= H - 1) continue;
        // vertices of the triangle: A=(X,Y), middle (B or D), C=(X+1,Y+1)
        const int mx = (t == 0) ? X + 1 : X, my = (t == 0) ? Y : Y + 1;
        const int vx[3] = {X, mx, X + 1}, vy[3] = {Y, my, Y + 1};
        R u[3][3], l[3][3], fa[3], fb[3];
        for (int i = 0; i < 3; ++i) {
            U.at(vx[i], vy[i], u[i]);
            L.at(vx[i], vy[i], l[i]);
            fa[i] = f1[(long long)vy[i] * pitch + vx[i]];
            fb[i] = f2[(long long)vy[i] * pitch + vx[i]];
        }
        R g[3];
        if (t == 0) { g[0] = fb[1] - fb[0]; g[1] = fb[2] - fb[1]; }
        else        { g[0] = fb[2] - fb[1]; g[1] = fb[1] - fb[0]; }
        g[2] = -(fa[0] + fa[1] + fa[2]) * third * gms;
        const R ft = ((fb[0] - fa[0]) + (fb[1] - fa[1]) + (fb[2] - fa[2])) * third;
        R dEdg[3], dEdft;
        elem_adjoint<R>(u, l, g, ft, dEdg, dEdft);
        a2 -= dEdg[0] * phx[e] + dEdg[1] * phy[e] + dEdft * third;
        a1 += (dEdg[2] * gms + dEdft) * third;
    }
    if (df2) df2[(long long)y * W + x] = (O)a2;
    if (df1) df1[(long long)y * W + x] = (O)a1;
}

// K_rho data term: per element (the 18 planes of the element data layout)
//   dE/dA_cd = |K|/12 (sum_i Lam_ic U_id + (sum_i Lam_ic)(sum_i U_id))   (c = d)
//   and its sum with the transpose for the stored off-diagonal entries,
//   dE/dF_c  = -|K|/3 sum_i Lam_ic.
template <typename R>
__global__ void k_adjoint_eld(const PairDesc* pairs, int pair, const double* __restrict__ ua,
                              const double* __restrict__ la, R* __restrict__ G, long long stride) {
    const PairDesc pd = pairs[pair];
    const int W = pd.W, H = pd.H, pitch = pd.pitch;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W - 1 || y >= H - 1) return;
    UView<double, double> U{ua + pd.vec_off, (long long)H * pitch, pitch};
    UView<double, double> L{la + pd.vec_off, (long long)H * pitch, pitch};
    double uA[3], uB[3], uC[3], uD[3], lA[3], lB[3], lC[3], lD[3];
    U.at(x, y, uA); U.at(x + 1, y, uB); U.at(x + 1, y + 1, uC); U.at(x, y + 1, uD);
    L.at(x, y, lA); L.at(x + 1, y, lB); L.at(x + 1, y + 1, lC); L.at(x, y + 1, lD);
    const double k12 = 0.5 / 12.0, k3 = 0.5 / 3.0;
    const int sc[6] = {0, 0, 0, 1, 1, 2}, sd[6] = {0, 1, 2, 1, 2, 2};
    R* g0 = G + pd.frame_off + (long long)y * pitch + x;
    for (int t = 0; t < 2; ++t) {
        const double* um = t == 0 ? uB : uD;
        const double* lm = t == 0 ? lB : lD;
        double M[3][3], Ls[3], Us[3];
        for (int c = 0; c < 3; ++c) {
            Ls[c] = lA[c] + lm[c] + lC[c];
            Us[c] = uA[c] + um[c] + uC[c];
        }
        for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d)
                M[c][d] = k12 * (lA[c] * uA[d] + lm[c] * um[d] + lC[c] * uC[d] + Ls[c] * Us[d]);
        R* gp = g0 + (long long)(9 * t) * stride;
        for (int k = 0; k < 6; ++k) {
            const int c = sc[k], d = sd[k];
            gp[k * stride] = (R)(c == d ? M[c][c] : M[c][d] + M[d][c]);
        }
        for (int c = 0; c < 3; ++c) gp[(6 + c) * stride] = (R)(-k3 * Ls[c]);
    }
}

// dL/df2, dL/df1 with K_rho: as k_adjoint_frames, but dE/dg and dE/dft of
// each element come from the K_rho^T-smoothed planes G of k_adjoint_eld:
//   dE/dg_m = sum_k G_k d(g_c g_d)/dg_m - ft G_F,m,   dE/dft = -sum_c G_F,c g_c.
template <typename R, typename O>
__global__ void k_adjoint_frames_eld(const PairDesc* pairs, int pair, const R* __restrict__ f1a,
                                     const R* __restrict__ f2a, const R* __restrict__ G, long long stride,
                                     O* __restrict__ df2, O* __restrict__ df1, double gms_d) {
    const PairDesc pd = pairs[pair];
    const R gms = (R)gms_d;
    const int W = pd.W, H = pd.H, pitch = pd.pitch;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    const R* f1 = f1a + pd.frame_off;
    const R* f2 = f2a + pd.frame_off;
    const int sqx[6] = {x, x, x - 1, x - 1, x - 1, x};
    const int sqy[6] = {y, y, y - 1, y - 1, y, y - 1};
    const int sqt[6] = {0, 1, 0, 1, 0, 1};
    const R phx[6] = {-1, 0, 0, 1, 1, -1};
    const R phy[6] = {0, -1, 1, 0, -1, 1};
    const R third = R(1) / R(3);
    R a2 = R(0), a1 = R(0);
    for (int e = 0; e < 6; ++e) {
        const int X = sqx[e], Y = sqy[e], t = sqt[e];
        if (X < 0 || Y < 0 || X >= W - 1 || Y >= H - 1) continue;
        const int mx = (t == 0) ? X + 1 : X, my = (t == 0) ? Y : Y + 1;
        const int vx[3] = {X, mx, X + 1}, vy[3] = {Y, my, Y + 1};
        R fa[3], fb[3];
        for (int i = 0; i < 3; ++i) {
            fa[i] = f1[(long long)vy[i] * pitch + vx[i]];
            fb[i] = f2[(long long)vy[i] * pitch + vx[i]];
        }
        R g[3];
        if (t == 0) { g[0] = fb[1] - fb[0]; g[1] = fb[2] - fb[1]; }
        else        { g[0] = fb[2] - fb[1]; g[1] = fb[1] - fb[0]; }
        g[2] = -(fa[0] + fa[1] + fa[2]) * third * gms;
        const R ft = ((fb[0] - fa[0]) + (fb[1] - fa[1]) + (fb[2] - fa[2])) * third;
        const R* gp = G + pd.frame_off + (long long)Y * pitch + X + (long long)(9 * t) * stride;
        R Ga[6], GF[3];
        for (int k = 0; k < 6; ++k) Ga[k] = gp[k * stride];
        for (int c = 0; c < 3; ++c) GF[c] = gp[(6 + c) * stride];
        // entries 00, 01, 02, 11, 12, 22
        R dEdg[3];
        dEdg[0] = R(2) * Ga[0] * g[0] + Ga[1] * g[1] + Ga[2] * g[2] - ft * GF[0];
        dEdg[1] = Ga[1] * g[0] + R(2) * Ga[3] * g[1] + Ga[4] * g[2] - ft * GF[1];
        dEdg[2] = Ga[2] * g[0] + Ga[4] * g[1] + R(2) * Ga[5] * g[2] - ft * GF[2];
        const R dEdft = -(GF[0] * g[0] + GF[1] * g[1] + GF[2] * g[2]);
        a2 -= dEdg[0] * phx[e] + dEdg[1] * phy[e] + dEdft * third;
        a1 += (dEdg[2] * gms + dEdft) * third;
    }
    if (df2) df2[(long long)y * W + x] = (O)a2;
    if (df1) df1[(long long)y * W + x] = (O)a1;
}

// Frame gradients from per-element planes G (the layout of the element data)
// holding minus the derivatives with respect to A_rho (6 stored entries) and F:
// K_rho^T over each plane, then k_adjoint_frames_eld.
template <typename R, typename O>
static cudaError_t eld_frames_chain(const AdaptBufs& A, int pair, int H, int W, void* df2, void* df1, int type,
                                    cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    const size_t es = sizeof(R);
    for (int q = 0; q < 18; ++q) {  // K_rho^T over each plane's (W-1) x (H-1) lattice
        e = launch_smooth((char*)A.eldg + ((size_t)q * A.eld_stride + A.frame_off) * es, A.scratch, type, W - 1, H - 1,
                          A.pitch, *A.taps_rho, true, st);
        if (e != cudaSuccess) return e;
    }
    dim3 gf((W + 127) / 128, H);
    k_adjoint_frames_eld<R, O><<<gf, 128, 0, st>>>(A.pairs, pair, (const R*)A.f1, (const R*)A.f2, (const R*)A.eldg,
                                                   A.eld_stride, (O*)df2, (O*)df1, A.gms);
    return cudaGetLastError();
}

template <typename R, typename O>
static cudaError_t adjoint_frames_eld(const AdaptBufs& A, int pair, int H, int W, const double* lamv, void* df2,
                                      void* df1, int type, cudaStream_t st) {
    dim3 ge((W - 1 + 127) / 128, H - 1);
    k_adjoint_eld<R><<<ge, 128, 0, st>>>(A.pairs, pair, A.u, lamv, (R*)A.eldg, A.eld_stride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return eld_frames_chain<R, O>(A, pair, H, W, df2, df1, type, st);
}

// ------------------------------------------ through the adaptation pass --
// Vector-Jacobian products of one adaptation pass (indicator, then alpha
// update) for dL/dalpha_new = v, in FP64.
//
// Update: alpha' = max(alpha / (1 + kappa s), alpha_th), s = max(eta / m -
// eta_thr, 0), m = max eta.  The flat branches (alpha' = alpha_th, s = 0)
// pass nothing; m passes sum_K dL/ds_K (-eta_K / m^2) to the first element
// that attains it.  w = dL/deta, da = dL/dalpha through the update.
template <typename R, typename O>
__global__ void k_update_vjp(const PairDesc* pairs, int pair, const R* __restrict__ ala, const R* __restrict__ etaa,
                             const unsigned long long* __restrict__ etamax_bits, const O* __restrict__ v,
                             O* __restrict__ da, double* __restrict__ wa, double kappa, double eta_thr,
                             double alpha_th, double* __restrict__ part, unsigned long long* __restrict__ argmax) {
    __shared__ double sh[32];
    const PairDesc pd = pairs[pair];
    const int W = pd.W, H = pd.H, pitch = pd.pitch;
    const R* al_p = ala + 2 * pd.frame_off;
    const R* eta_p = etaa + 2 * pd.frame_off;
    double* w = wa + 2 * pd.frame_off;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const double m = __longlong_as_double((long long)etamax_bits[pair]);
    double acc = 0.0;
    if (x < W - 1 && y < H - 1) {
        for (int t = 0; t < 2; ++t) {
            const long long o = 2 * ((long long)y * pitch + x) + t;        // workspace layout
            const long long od = 2 * ((long long)y * (W - 1) + x) + t;     // dense [H-1][W-1][2]
            const double vv = (double)v[od];
            if (!(m > 0.0)) {  // no update happened: identity
                da[od] = (O)vv;
                w[o] = 0.0;
                continue;
            }
            const double eta = (double)eta_p[o], al = (double)al_p[o];
            const double rel = eta / m - eta_thr;
            const bool pos = rel > 0.0;
            const double den = 1.0 + kappa * (pos ? rel : 0.0);
            const bool active = al / den > alpha_th;
            da[od] = (O)(active ? vv / den : 0.0);
            const double ds = active ? -vv * al * kappa / (den * den) : 0.0;
            w[o] = pos ? ds / m : 0.0;
            if (pos) acc += ds * eta / (m * m);
            if (eta == m) atomicMin(argmax, (unsigned long long)(((long long)y * (W - 1) + x) * 2 + t));
        }
    }
    acc = block_sum<128>(acc, sh);
    if (threadIdx.x == 0) part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

// the max(eta) term: w[argmax] -= sum of the block partials (fixed order)
__global__ void k_update_vjp_max(const PairDesc* pairs, int pair, const unsigned long long* __restrict__ etamax_bits,
                                 const double* __restrict__ part, int nparts,
                                 const unsigned long long* __restrict__ argmax, double* __restrict__ wa) {
    __shared__ double sh[32];
    const PairDesc pd = pairs[pair];
    const double m = __longlong_as_double((long long)etamax_bits[pair]);
    const double s = ordered_sum<256>(part, nparts, 1, sh);
    const unsigned long long ne = 2ULL * (pd.W - 1) * (pd.H - 1);
    if (threadIdx.x == 0 && m > 0.0 && *argmax < ne) {
        const unsigned long long e = *argmax, sq = e >> 1;
        const int t = (int)(e & 1), x = (int)(sq % (pd.W - 1)), y = (int)(sq / (pd.W - 1));
        wa[2 * (pd.frame_off + (long long)y * pd.pitch + x) + t] -= s;
    }
}

// Indicator: per element K, its share of sum_K' w_K' eta_K' with respect to
// its own unknowns (Eq. errind as the forward kernel reads it):
//   interior  sqrt(2 integ), integ = G sum_a s_a^2 / 6:  d/dU of its vertices,
//             d/dalpha_K through G, d/dg and d/dft;
//   each edge 1/2 h_e sqrt(q_e) appears in the indicators of both elements
//             that share it, so with c_e = (w_K + w_O) h_e / (4 sqrt(q_e))
//             each side differentiates q_e with respect to its own flux
//             (J = out - in) and its own alpha (in J and in Lambda_e = max,
//             half the derivative to each side at a tie).
// Writes per element and triangle 13 values: dL/dU at its 3 vertices (3
// components each) and (dg_0, dg_1, dg_2, dft); adds dL/dalpha_K to da.
//
// With the K_rho element data (eld non-null) the interior residual at the
// edge midpoints m_a is R_a = F - A_rho U_h(m_a) and
//   integ = (|K|/3) sum_a sum_c R_ac^2 / Lambda_c,  d integ / d R_ac = R_ac / (3 Lambda_c);
// R_a is linear in F, in A_rho (-U_h(m_a)) and in the midpoint values
// (-A_rho).  The derivatives with respect to the element data go to eldg
// with a minus sign (the convention of k_adjoint_eld, so that the same K_rho^T
// chain to the frames serves both) and (dg, dft) are 0.
template <typename R, typename O>
__global__ void k_eta_vjp(const PairDesc* pairs, int pair, const R* __restrict__ f1a, const R* __restrict__ f2a,
                          const R* __restrict__ ala, const double* __restrict__ ua, const double* __restrict__ w,
                          double lam, double gms, O* __restrict__ da, double* __restrict__ buf, long long stride,
                          const R* __restrict__ eld, R* __restrict__ eldg) {
    const PairDesc pd = pairs[pair];
    const int W = pd.W, H = pd.H, pitch = pd.pitch;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W - 1 || y >= H - 1) return;
    const R* f1 = f1a + pd.frame_off;
    const R* f2 = f2a + pd.frame_off;
    const R* al = ala + 2 * pd.frame_off;
    const double* wp = w + 2 * pd.frame_off;
    UView<double, double> U{ua + pd.vec_off, (long long)H * pitch, pitch};
    auto F1 = [&](int xx, int yy) { return (double)f1[(long long)yy * pitch + xx]; };
    auto F2 = [&](int xx, int yy) { return (double)f2[(long long)yy * pitch + xx]; };
    auto AL = [&](int xx, int yy, int t) { return (double)al[2 * ((long long)yy * pitch + xx) + t]; };
    auto WW = [&](int xx, int yy, int t) { return wp[2 * ((long long)yy * pitch + xx) + t]; };
    double uA[3], uB[3], uC[3], uD[3];
    U.at(x, y, uA); U.at(x + 1, y, uB); U.at(x + 1, y + 1, uC); U.at(x, y + 1, uD);
    double gxK[2][3], gyK[2][3];
    tri_grad<double>(0, uA, uB, uC, uD, gxK[0], gyK[0]);
    tri_grad<double>(1, uA, uB, uC, uD, gxK[1], gyK[1]);
    const double third = 1.0 / 3.0, r2 = 0.7071067811865476, sq2 = 1.4142135623730951;
    // basis gradients of the vertices (A, B or D, C) of each family
    const double phx[2][3] = {{-1, 1, 0}, {0, -1, 1}}, phy[2][3] = {{0, -1, 1}, {-1, 1, 0}};
    for (int t = 0; t < 2; ++t) {
        const double* V[3] = {uA, t == 0 ? uB : uD, uC};
        double g[3], ft;
        if (t == 0) {
            g[0] = F2(x + 1, y) - F2(x, y); g[1] = F2(x + 1, y + 1) - F2(x + 1, y);
            g[2] = -(F1(x, y) + F1(x + 1, y) + F1(x + 1, y + 1)) * third * gms;
            ft = ((F2(x, y) - F1(x, y)) + (F2(x + 1, y) - F1(x + 1, y)) + (F2(x + 1, y + 1) - F1(x + 1, y + 1))) * third;
        } else {
            g[0] = F2(x + 1, y + 1) - F2(x, y + 1); g[1] = F2(x, y + 1) - F2(x, y);
            g[2] = -(F1(x, y) + F1(x, y + 1) + F1(x + 1, y + 1)) * third * gms;
            ft = ((F2(x, y) - F1(x, y)) + (F2(x, y + 1) - F1(x, y + 1)) + (F2(x + 1, y + 1) - F1(x + 1, y + 1))) * third;
        }
        const double aK = AL(x, y, t);
        const double LK[3] = {aK, aK, lam};
        const double wK = WW(x, y, t);
        double dU[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, dg[3] = {0, 0, 0}, dft = 0.0, dal = 0.0;
        double um[3][3];
        for (int a = 0; a < 3; ++a) {
            const int b = (a + 1) % 3;
            for (int c = 0; c < 3; ++c) um[a][c] = 0.5 * (V[a][c] + V[b][c]);
        }
        // interior
        if (eld) {
            const long long eo = pd.frame_off + (long long)y * pitch + x + (long long)(9 * t) * stride;
            double A6[6], F[3];
            for (int k = 0; k < 6; ++k) A6[k] = (double)eld[eo + k * stride];
            for (int c = 0; c < 3; ++c) F[c] = (double)eld[eo + (6 + c) * stride];
            const double Am[3][3] = {{A6[0], A6[1], A6[2]}, {A6[1], A6[3], A6[4]}, {A6[2], A6[4], A6[5]}};
            double Rr[3][3], integ = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                    Rr[a][c] = F[c] - (Am[c][0] * um[a][0] + Am[c][1] * um[a][1] + Am[c][2] * um[a][2]);
                    integ += Rr[a][c] * Rr[a][c] / LK[c];
                }
            integ *= 0.5 / 3.0;
            const double wi = integ > 0.0 ? wK / sqrt(2.0 * integ) : 0.0;
            double GA[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, GF[3] = {0, 0, 0};
            for (int a = 0; a < 3; ++a) {
                const int b = (a + 1) % 3;
                double dR[3];
                for (int c = 0; c < 3; ++c) {
                    dR[c] = wi * Rr[a][c] / (3.0 * LK[c]);
                    GF[c] += dR[c];
                }
                for (int c = 0; c < 3; ++c)
                    for (int d = 0; d < 3; ++d) GA[c][d] -= dR[c] * um[a][d];
                for (int d = 0; d < 3; ++d) {
                    const double dum = -(Am[0][d] * dR[0] + Am[1][d] * dR[1] + Am[2][d] * dR[2]);
                    dU[a][d] += 0.5 * dum;
                    dU[b][d] += 0.5 * dum;
                }
                dal += wi * (0.5 / 3.0) * (-(Rr[a][0] * Rr[a][0] + Rr[a][1] * Rr[a][1]) / (aK * aK));
            }
            // entries 00, 01, 02, 11, 12, 22, then F; negated (see above)
            R* gp = eldg + eo;
            gp[0] = (R)(-GA[0][0]);
            gp[stride] = (R)(-(GA[0][1] + GA[1][0]));
            gp[2 * stride] = (R)(-(GA[0][2] + GA[2][0]));
            gp[3 * stride] = (R)(-GA[1][1]);
            gp[4 * stride] = (R)(-(GA[1][2] + GA[2][1]));
            gp[5 * stride] = (R)(-GA[2][2]);
            for (int c = 0; c < 3; ++c) gp[(6 + c) * stride] = (R)(-GF[c]);
        } else {
            const double G = g[0] * g[0] / LK[0] + g[1] * g[1] / LK[1] + g[2] * g[2] / LK[2];
            double s[3], S2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                s[a] = ft + g[0] * um[a][0] + g[1] * um[a][1] + g[2] * um[a][2];
                S2 += s[a] * s[a];
            }
            const double integ = G * S2 / 6.0;
            const double wi = integ > 0.0 ? wK / sqrt(2.0 * integ) : 0.0;
            for (int a = 0; a < 3; ++a) {
                const int b = (a + 1) % 3;
                const double k = wi * G * s[a] / 3.0;
                for (int c = 0; c < 3; ++c) {
                    dU[a][c] += 0.5 * k * g[c];
                    dU[b][c] += 0.5 * k * g[c];
                    dg[c] += k * um[a][c];
                }
                dft += k;
            }
            for (int c = 0; c < 3; ++c) dg[c] += wi * S2 / 6.0 * 2.0 * g[c] / LK[c];
            dal += wi * S2 / 6.0 * (-(g[0] * g[0] + g[1] * g[1]) / (aK * aK));
        }
        // edges
        double dgx[3] = {0, 0, 0}, dgy[3] = {0, 0, 0};  // dL/d(grad U_c) of this element
        for (int e = 0; e < 3; ++e) {
            double nx, ny, he;
            int nbx = 0, nby = 0, nbt = 0;
            bool has;
            if (t == 0) {
                if (e == 0) { nx = 0; ny = -1; he = 1; has = y >= 1; nbx = x; nby = y - 1; nbt = 1; }
                else if (e == 1) { nx = 1; ny = 0; he = 1; has = x + 1 <= W - 2; nbx = x + 1; nby = y; nbt = 1; }
                else { nx = -r2; ny = r2; he = sq2; has = true; nbx = x; nby = y; nbt = 1; }
            } else {
                if (e == 0) { nx = -1; ny = 0; he = 1; has = x >= 1; nbx = x - 1; nby = y; nbt = 0; }
                else if (e == 1) { nx = 0; ny = 1; he = 1; has = y + 1 <= H - 2; nbx = x; nby = y + 1; nbt = 0; }
                else { nx = r2; ny = -r2; he = sq2; has = true; nbx = x; nby = y; nbt = 0; }
            }
            double ngx[3] = {0, 0, 0}, ngy[3] = {0, 0, 0}, aO = 0.0, wO = 0.0;
            if (has) {
                if (nbx == x && nby == y) {
                    for (int c = 0; c < 3; ++c) { ngx[c] = gxK[nbt][c]; ngy[c] = gyK[nbt][c]; }
                } else {
                    double qA[3], qB[3], qC[3], qD[3];
                    U.at(nbx, nby, qA); U.at(nbx + 1, nby, qB); U.at(nbx + 1, nby + 1, qC); U.at(nbx, nby + 1, qD);
                    tri_grad<double>(nbt, qA, qB, qC, qD, ngx, ngy);
                }
                aO = AL(nbx, nby, nbt);
                wO = WW(nbx, nby, nbt);
            }
            double J[3], Le[3], q = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double lo = c < 2 ? aO : lam;
                const double fin = LK[c] * (gxK[t][c] * nx + gyK[t][c] * ny);
                const double fout = has ? lo * (ngx[c] * nx + ngy[c] * ny) : 0.0;
                Le[c] = has ? (lo > LK[c] ? lo : LK[c]) : LK[c];
                J[c] = fout - fin;
                q += J[c] * J[c] / Le[c];
            }
            const double wt = wK + (has ? wO : 0.0);
            const double ce = q > 0.0 ? wt * 0.25 * he / sqrt(q) : 0.0;
            for (int c = 0; c < 3; ++c) {
                const double dJ = ce * 2.0 * J[c] / Le[c];
                dgx[c] += -LK[c] * dJ * nx;
                dgy[c] += -LK[c] * dJ * ny;
                if (c < 2) {
                    const double share = has ? (LK[c] > aO ? 1.0 : (LK[c] == aO ? 0.5 : 0.0)) : 1.0;
                    dal += dJ * (-(gxK[t][c] * nx + gyK[t][c] * ny)) + ce * (-(J[c] * J[c]) / (Le[c] * Le[c])) * share;
                }
            }
        }
        for (int i = 0; i < 3; ++i)
            for (int c = 0; c < 3; ++c) dU[i][c] += phx[t][i] * dgx[c] + phy[t][i] * dgy[c];
        double* bp = buf + pd.frame_off + (long long)y * pitch + x + (long long)(13 * t) * stride;
        for (int i = 0; i < 3; ++i)
            for (int c = 0; c < 3; ++c) bp[(3 * i + c) * stride] = dU[i][c];
        for (int c = 0; c < 3; ++c) bp[(9 + c) * stride] = dg[c];
        bp[12 * stride] = dft;
        const long long od = 2 * ((long long)y * (W - 1) + x) + t;
        da[od] = (O)((double)da[od] + dal);
    }
}

// per node: dL/dU (its 6 elements' vertex values) and dL/df2, dL/df1 (the
// frame chain of their (dg, dft)), dense [3][H][W] and [H][W] outputs
template <typename O>
__global__ void k_eta_vjp_nodes(const PairDesc* pairs, int pair, const double* __restrict__ buf, long long stride,
                                double gms, O* __restrict__ dU, O* __restrict__ df2, O* __restrict__ df1) {
    const PairDesc pd = pairs[pair];
    const int W = pd.W, H = pd.H, pitch = pd.pitch;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W) return;
    // E1 sq(x,y).t0 vertex 0, E2 sq(x,y).t1 vertex 0, E3 sq(x-1,y-1).t0 vertex 2,
    // E4 sq(x-1,y-1).t1 vertex 2, E5 sq(x-1,y).t0 vertex 1, E6 sq(x,y-1).t1 vertex 1
    const int sqx[6] = {x, x, x - 1, x - 1, x - 1, x};
    const int sqy[6] = {y, y, y - 1, y - 1, y, y - 1};
    const int sqt[6] = {0, 1, 0, 1, 0, 1};
    const int vtx[6] = {0, 0, 2, 2, 1, 1};
    const double phx[6] = {-1, 0, 0, 1, 1, -1};
    const double phy[6] = {0, -1, 1, 0, -1, 1};
    double u[3] = {0, 0, 0}, a2 = 0.0, a1 = 0.0;
    for (int e = 0; e < 6; ++e) {
        const int X = sqx[e], Y = sqy[e], t = sqt[e];
        if (X < 0 || Y < 0 || X >= W - 1 || Y >= H - 1) continue;
        const double* bp = buf + pd.frame_off + (long long)Y * pitch + X + (long long)(13 * t) * stride;
        for (int c = 0; c < 3; ++c) u[c] += bp[(3 * vtx[e] + c) * stride];
        const double dg0 = bp[9 * stride], dg1 = bp[10 * stride], dg2 = bp[11 * stride], dft = bp[12 * stride];
        a2 += dg0 * phx[e] + dg1 * phy[e] + dft / 3.0;
        a1 += -gms * dg2 / 3.0 - dft / 3.0;
    }
    const long long o = (long long)y * W + x, plane = (long long)H * W;
    if (dU) { dU[o] = (O)u[0]; dU[o + plane] = (O)u[1]; dU[o + 2 * plane] = (O)u[2]; }
    if (df2) df2[o] = (O)a2;
    if (df1) df1[o] = (O)a1;
}

template <typename R, typename O>
static cudaError_t adapt_vjp_t(const AdaptBufs& A, int pair, int H, int W, double kappa, double eta_thr,
                               double alpha_th, const void* v, void* da, void* dU, void* df2, void* df1,
                               cudaStream_t st) {
    const dim3 ge((W - 1 + 127) / 128, H - 1);
    const int nparts = (int)(ge.x * ge.y);
    cudaError_t e = cudaMemsetAsync(A.vjp_argmax, 0xff, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_update_vjp<R, O><<<ge, 128, 0, st>>>(A.pairs, pair, (const R*)A.alpha, (const R*)A.eta,
                                           (const unsigned long long*)A.etamax, (const O*)v, (O*)da, A.vjp_w, kappa,
                                           eta_thr, alpha_th, A.vjp_part, A.vjp_argmax);
    k_update_vjp_max<<<1, 256, 0, st>>>(A.pairs, pair, (const unsigned long long*)A.etamax, A.vjp_part, nparts,
                                        A.vjp_argmax, A.vjp_w);
    const bool eldm = A.eld != nullptr;  // K_rho: the frame chain goes through the element data
    k_eta_vjp<R, O><<<ge, 128, 0, st>>>(A.pairs, pair, (const R*)A.f1, (const R*)A.f2, (const R*)A.alpha, A.u,
                                        A.vjp_w, A.lam, A.gms, (O*)da, A.vjp_buf, A.eld_stride,
                                        eldm ? (const R*)A.eld : nullptr, eldm ? (R*)A.eldg : nullptr);
    const dim3 gn((W + 127) / 128, H);
    k_eta_vjp_nodes<O><<<gn, 128, 0, st>>>(A.pairs, pair, A.vjp_buf, A.eld_stride, A.gms, (O*)dU,
                                           eldm ? nullptr : (O*)df2, eldm ? nullptr : (O*)df1);
    e = cudaGetLastError();
    if (e != cudaSuccess || !eldm || !(df2 || df1)) return e;
    return eld_frames_chain<R, O>(A, pair, H, W, df2, df1, A.fp64 ? T_F64 : T_F32, st);
}

cudaError_t launch_adapt_vjp(const AdaptBufs& A, int pair, int H, int W, double kappa, double eta_thr,
                             double alpha_th, const void* v, void* da, void* dU, void* df2, void* df1, int out_type,
                             cudaStream_t st) {
    if (A.fp64)
        return out_type == T_F64 ? adapt_vjp_t<double, double>(A, pair, H, W, kappa, eta_thr, alpha_th, v, da, dU, df2, df1, st)
                                 : adapt_vjp_t<double, float>(A, pair, H, W, kappa, eta_thr, alpha_th, v, da, dU, df2, df1, st);
    return out_type == T_F64 ? adapt_vjp_t<float, double>(A, pair, H, W, kappa, eta_thr, alpha_th, v, da, dU, df2, df1, st)
                             : adapt_vjp_t<float, float>(A, pair, H, W, kappa, eta_thr, alpha_th, v, da, dU, df2, df1, st);
}

cudaError_t launch_adjoint_grad(const AdaptBufs& A, int pair, int H, int W, const double* lamv, void* dalpha,
                                void* df2, void* df1, int out_type, cudaStream_t st) {
    if (dalpha) {
        dim3 grid((W - 1 + 127) / 128, H - 1);
        if (A.fp64) {
            if (out_type == T_F64) k_adjoint_alpha<double, double><<<grid, 128, 0, st>>>(A.pairs, pair, A.u, lamv, (double*)dalpha);
            else k_adjoint_alpha<double, float><<<grid, 128, 0, st>>>(A.pairs, pair, A.u, lamv, (float*)dalpha);
        } else {
            if (out_type == T_F64) k_adjoint_alpha<float, double><<<grid, 128, 0, st>>>(A.pairs, pair, A.u, lamv, (double*)dalpha);
            else k_adjoint_alpha<float, float><<<grid, 128, 0, st>>>(A.pairs, pair, A.u, lamv, (float*)dalpha);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if ((df2 || df1) && A.eld) {
        if (A.fp64)
            return out_type == T_F64 ? adjoint_frames_eld<double, double>(A, pair, H, W, lamv, df2, df1, T_F64, st)
                                     : adjoint_frames_eld<double, float>(A, pair, H, W, lamv, df2, df1, T_F64, st);
        return out_type == T_F64 ? adjoint_frames_eld<float, double>(A, pair, H, W, lamv, df2, df1, T_F32, st)
                                 : adjoint_frames_eld<float, float>(A, pair, H, W, lamv, df2, df1, T_F32, st);
    }
    if (df2 || df1) {
        dim3 grid((W + 127) / 128, H);
        if (A.fp64) {
            if (out_type == T_F64)
                k_adjoint_frames<double, double><<<grid, 128, 0, st>>>(A.pairs, pair, (const double*)A.f1, (const double*)A.f2, A.u, lamv, (double*)df2, (double*)df1, A.gms);
            else
                k_adjoint_frames<double, float><<<grid, 128, 0, st>>>(A.pairs, pair, (const double*)A.f1, (const double*)A.f2, A.u, lamv, (float*)df2, (float*)df1, A.gms);
        } else {
            if (out_type == T_F64)
                k_adjoint_frames<float, double><<<grid, 128, 0, st>>>(A.pairs, pair, (const float*)A.f1, (const float*)A.f2, A.u, lamv, (double*)df2, (double*)df1, A.gms);
            else
                k_adjoint_frames<float, float><<<grid, 128, 0, st>>>(A.pairs, pair, (const float*)A.f1, (const float*)A.f2, A.u, lamv, (float*)df2, (float*)df1, A.gms);
        }
    }
    return cudaGetLastError();
}

}  // namespace ofl
