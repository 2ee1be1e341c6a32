// Matrix-free apply of the P1 operator of Section 2.2 (Eq. discret-form),
// element by element, streamed down pixel columns.
//
// Layout of the work: a warp owns 32 consecutive square columns; lane l
// computes the two triangles of square (cx, sy) for cx = X0 + 31 w - 1 + l
// while walking down the rows.  The 4 corner contributions of a square are
// combined across lanes with one shuffle (left corners of square cx+1 come
// from lane l+1) and across rows with a register carry (top corners of row
// sy are the bottom corners' partners of row sy+1), so every element is
// formed exactly once and every input word is read once per warp (plus a
// one-column halo).  Lane 31 only helps: each warp outputs 31 columns.
//
// Modes (template MODE):
//   APPLY : out = A in                                  (+ optional load b)
//   PCG   : in = z + beta p_old  (p_new stored),  d += a_prev p_old,
//           out q = A in,  partial sum p.q  -> pair scalar a = rz / pq
//   RES   : in = x + d + a p  (x_new stored),  out r = rhs - A in,
//           rhs = b (frames) or a given vector,  partial ||r||^2, ||rhs||^2
#pragma once
#include <type_traits>

#include "of_common.cuh"
#include "of_df.cuh"

namespace ofk {

enum { MODE_APPLY = 0, MODE_PCG = 1, MODE_RES = 2, MODE_RESB = 3 };
// MODE_RESB: MODE_RES for x = 0 (cold start): r = rhs, only the load is formed.

template <typename R> struct V3 { R a, b, c; };
template <typename R> __device__ __forceinline__ V3<R> v3(R a, R b, R c) { V3<R> v; v.a = a; v.b = b; v.c = c; return v; }
template <typename R> __device__ __forceinline__ V3<R> operator+(V3<R> x, V3<R> y) { return v3(x.a + y.a, x.b + y.b, x.c + y.c); }
template <typename R> __device__ __forceinline__ V3<R> shfl_down3(V3<R> x) { return v3(shfl_down(x.a, 1), shfl_down(x.b, 1), shfl_down(x.c, 1)); }

template <typename R> struct NodeVal { V3<R> p; R f1, f2; };

// Contributions of the two triangles of one square to its corners
// A=(x,y) B=(x+1,y) C=(x+1,y+1) D=(x,y+1): sign * (A_K p)_i, and, when WANT_B,
// the load -|K|/3 ft g of each triangle (same for its 3 vertices).  gms
// scales the illumination column g_m of the element data: 1 for the model
// with brightness change, 0 for brightness constancy.
template <typename R, bool WANT_B, bool WANT_A = true>
__device__ __forceinline__ void square_contrib(const NodeVal<R>& A, const NodeVal<R>& B, const NodeVal<R>& C,
                                               const NodeVal<R>& D, R al0, R al1, R lam, R gms, bool valid,
                                               V3<R>& cA, V3<R>& cB, V3<R>& cC, V3<R>& cD,
                                               V3<R>& bA, V3<R>& bB, V3<R>& bC, V3<R>& bD) {
    constexpr R third = kconst<R>(1.0 / 3.0);
    constexpr R w24 = kconst<R>(1.0 / 24.0);
    constexpr R h = kconst<R>(OF_STIFF_HALF);
    constexpr R zero = kconst<R>(0.0);
    // ---- t = 0: A, B, C
    R g0x = B.f2 - A.f2, g0y = C.f2 - B.f2, g0m = -(A.f1 + B.f1 + C.f1) * third * gms;
    R g1x = C.f2 - D.f2, g1y = D.f2 - A.f2, g1m = -(A.f1 + D.f1 + C.f1) * third * gms;
    if constexpr (!WANT_A) {
        cA = cB = cC = cD = v3(zero, zero, zero);
    } else {
    R sA = g0x * A.p.a + g0y * A.p.b + g0m * A.p.c;
    R sB = g0x * B.p.a + g0y * B.p.b + g0m * B.p.c;
    R sC = g0x * C.p.a + g0y * C.p.b + g0m * C.p.c;
    R S0 = sA + sB + sC;
    R wA = (sA + S0) * w24, wB = (sB + S0) * w24, wC = (sC + S0) * w24;
    // ---- t = 1: A, D, C
    R tA = g1x * A.p.a + g1y * A.p.b + g1m * A.p.c;
    R tD = g1x * D.p.a + g1y * D.p.b + g1m * D.p.c;
    R tC = g1x * C.p.a + g1y * C.p.b + g1m * C.p.c;
    R S1 = tA + tD + tC;
    R vA = (tA + S1) * w24, vD = (tD + S1) * w24, vC = (tC + S1) * w24;
    // stiffness: legs A-B, B-C (t=0) and A-D, D-C (t=1), weight 1/2 each
    R a0 = h * al0, a1 = h * al1, l0 = h * lam;
    V3<R> dAB = v3(A.p.a - B.p.a, A.p.b - B.p.b, A.p.c - B.p.c);
    V3<R> dCB = v3(C.p.a - B.p.a, C.p.b - B.p.b, C.p.c - B.p.c);
    V3<R> dAD = v3(A.p.a - D.p.a, A.p.b - D.p.b, A.p.c - D.p.c);
    V3<R> dCD = v3(C.p.a - D.p.a, C.p.b - D.p.b, C.p.c - D.p.c);
    cA.a = wA * g0x + vA * g1x + a0 * dAB.a + a1 * dAD.a;
    cA.b = wA * g0y + vA * g1y + a0 * dAB.b + a1 * dAD.b;
    cA.c = wA * g0m + vA * g1m + l0 * (dAB.c + dAD.c);
    cB.a = wB * g0x - a0 * (dAB.a + dCB.a);
    cB.b = wB * g0y - a0 * (dAB.b + dCB.b);
    cB.c = wB * g0m - l0 * (dAB.c + dCB.c);
    cC.a = wC * g0x + vC * g1x + a0 * dCB.a + a1 * dCD.a;
    cC.b = wC * g0y + vC * g1y + a0 * dCB.b + a1 * dCD.b;
    cC.c = wC * g0m + vC * g1m + l0 * (dCB.c + dCD.c);
    cD.a = vD * g1x - a1 * (dAD.a + dCD.a);
    cD.b = vD * g1y - a1 * (dAD.b + dCD.b);
    cD.c = vD * g1m - l0 * (dAD.c + dCD.c);
    }
    if constexpr (WANT_B) {
        constexpr R sixth = kconst<R>(1.0 / 6.0);
        R ft0 = ((A.f2 - A.f1) + (B.f2 - B.f1) + (C.f2 - C.f1)) * third;
        R ft1 = ((A.f2 - A.f1) + (D.f2 - D.f1) + (C.f2 - C.f1)) * third;
        R k0 = -sixth * ft0, k1 = -sixth * ft1;
        V3<R> b0 = v3(k0 * g0x, k0 * g0y, k0 * g0m);
        V3<R> b1 = v3(k1 * g1x, k1 * g1y, k1 * g1m);
        bA = b0 + b1; bB = b0; bC = b0 + b1; bD = b1;
    }
    if (!valid) {
        cA = cB = cC = cD = v3(zero, zero, zero);
        if constexpr (WANT_B) bA = bB = bC = bD = v3(zero, zero, zero);
    }
}

// square_contrib with a per-element lambda (lam0 on t = 0, lam1 on t = 1)
// instead of the constant: the m stiffness is added per triangle.
template <typename R, bool WANT_B, bool WANT_A = true>
__device__ __forceinline__ void square_contrib_l(const NodeVal<R>& A, const NodeVal<R>& B, const NodeVal<R>& C,
                                                 const NodeVal<R>& D, R al0, R al1, R lam0, R lam1, R gms, bool valid,
                                                 V3<R>& cA, V3<R>& cB, V3<R>& cC, V3<R>& cD,
                                                 V3<R>& bA, V3<R>& bB, V3<R>& bC, V3<R>& bD) {
    constexpr R zero = kconst<R>(0.0);
    square_contrib<R, WANT_B, WANT_A>(A, B, C, D, al0, al1, zero, gms, valid, cA, cB, cC, cD, bA, bB, bC, bD);
    if constexpr (WANT_A) {
        if (valid) {
            constexpr R h = kconst<R>(OF_STIFF_HALF);
            const R l0 = h * lam0, l1 = h * lam1;
            const R dAB = A.p.c - B.p.c, dCB = C.p.c - B.p.c, dAD = A.p.c - D.p.c, dCD = C.p.c - D.p.c;
            cA.c = cA.c + (l0 * dAB + l1 * dAD);
            cB.c = cB.c - l0 * (dAB + dCB);
            cC.c = cC.c + (l0 * dCB + l1 * dCD);
            cD.c = cD.c - l1 * (dAD + dCD);
        }
    }
}

// The same with general element data (K_rho > 0): per triangle the tensor
// A (entries 00, 01, 02, 11, 12, 22) and the load vector F of Section 1.
// Data term of vertex i: |K|/12 A (p_i + sum_j p_j); load |K|/3 F.
template <typename R>
__device__ __forceinline__ V3<R> sym_mv(const R* a, R x, R y, R z) {
    return v3(a[0] * x + a[1] * y + a[2] * z, a[1] * x + a[3] * y + a[4] * z, a[2] * x + a[4] * y + a[5] * z);
}

template <typename R, bool WANT_B, bool WANT_A = true>
__device__ __forceinline__ void square_contrib_el(const V3<R>& pA, const V3<R>& pB, const V3<R>& pC, const V3<R>& pD,
                                                  R al0, R al1, R lam, const R (&e0)[9], const R (&e1)[9], bool valid,
                                                  V3<R>& cA, V3<R>& cB, V3<R>& cC, V3<R>& cD, V3<R>& bA,
                                                  V3<R>& bB, V3<R>& bC, V3<R>& bD) {
    constexpr R w24 = kconst<R>(1.0 / 24.0);
    constexpr R h = kconst<R>(OF_STIFF_HALF);
    constexpr R zero = kconst<R>(0.0);
    if constexpr (!WANT_A) {
        cA = cB = cC = cD = v3(zero, zero, zero);
    } else {
        // t = 0: A, B, C
        const V3<R> S0 = pA + pB + pC;
        const V3<R> uA = pA + S0, uB = pB + S0, uC = pC + S0;
        const V3<R> wA = sym_mv(e0, uA.a * w24, uA.b * w24, uA.c * w24);
        const V3<R> wB = sym_mv(e0, uB.a * w24, uB.b * w24, uB.c * w24);
        const V3<R> wC = sym_mv(e0, uC.a * w24, uC.b * w24, uC.c * w24);
        // t = 1: A, D, C
        const V3<R> S1 = pA + pD + pC;
        const V3<R> tA = pA + S1, tD = pD + S1, tC = pC + S1;
        const V3<R> vA = sym_mv(e1, tA.a * w24, tA.b * w24, tA.c * w24);
        const V3<R> vD = sym_mv(e1, tD.a * w24, tD.b * w24, tD.c * w24);
        const V3<R> vC = sym_mv(e1, tC.a * w24, tC.b * w24, tC.c * w24);
        // stiffness as in square_contrib
        R a0 = h * al0, a1 = h * al1, l0 = h * lam;
        V3<R> dAB = v3(pA.a - pB.a, pA.b - pB.b, pA.c - pB.c);
        V3<R> dCB = v3(pC.a - pB.a, pC.b - pB.b, pC.c - pB.c);
        V3<R> dAD = v3(pA.a - pD.a, pA.b - pD.b, pA.c - pD.c);
        V3<R> dCD = v3(pC.a - pD.a, pC.b - pD.b, pC.c - pD.c);
        cA.a = wA.a + vA.a + a0 * dAB.a + a1 * dAD.a;
        cA.b = wA.b + vA.b + a0 * dAB.b + a1 * dAD.b;
        cA.c = wA.c + vA.c + l0 * (dAB.c + dAD.c);
        cB.a = wB.a - a0 * (dAB.a + dCB.a);
        cB.b = wB.b - a0 * (dAB.b + dCB.b);
        cB.c = wB.c - l0 * (dAB.c + dCB.c);
        cC.a = wC.a + vC.a + a0 * dCB.a + a1 * dCD.a;
        cC.b = wC.b + vC.b + a0 * dCB.b + a1 * dCD.b;
        cC.c = wC.c + vC.c + l0 * (dCB.c + dCD.c);
        cD.a = vD.a - a1 * (dAD.a + dCD.a);
        cD.b = vD.b - a1 * (dAD.b + dCD.b);
        cD.c = vD.c - l0 * (dAD.c + dCD.c);
    }
    if constexpr (WANT_B) {
        constexpr R sixth = kconst<R>(1.0 / 6.0);
        V3<R> b0 = v3(sixth * e0[6], sixth * e0[7], sixth * e0[8]);
        V3<R> b1 = v3(sixth * e1[6], sixth * e1[7], sixth * e1[8]);
        bA = b0 + b1; bB = b0; bC = b0 + b1; bD = b1;
    }
    if (!valid) {
        cA = cB = cC = cD = v3(zero, zero, zero);
        if constexpr (WANT_B) bA = bB = bC = bD = v3(zero, zero, zero);
    }
}

template <typename R, typename C, typename RI>
struct ApplyParams {
    const PairDesc* pairs;
    const int4* blocks;        // per block: (pair, column block, row block, global block index)
    const PairScalars* sc_in;  // PCG: beta, a_prev, it; RES: a
    PairScalars* sc;           // scalars written by the last block
    double* partial;           // [nblocks][2]
    unsigned* counter;         // [batch]
    unsigned* gcounter;        // [blocks]: FP32 PCG apply, arrivals of each group of 32 blocks (at its first block)
    int pq_fixed;              // FP32 PCG apply, one pair: p.q into PairScalars::pq_fix, a formed by the preconditioner
    const C* f1; const C* f2; const C* alpha;
    const C* lamel;            // per-element lambda [H][pitch][2] like alpha, or null (the constant lam)
    R lam;
    R gms;                     // illumination column scale (1: model with m, 0: brightness constancy)
    const C* eld;              // K_rho element data: 18 planes (t * 9 + k), plane stride eld_stride
    long long eld_stride;
    int rows_per_block;
    // vectors ([3][H][pitch] planes at pair vec_off)
    const R* in;        // APPLY: p;  PCG: z;  RES: x (double)
    RI* p_buf0;         // PCG: p buffers (even / odd);  RES: p buffers of the inner solve
    RI* p_buf1;
    RI* dcorr;          // PCG: d (in/out);  RES: d (in)
    R* out;             // APPLY: q; PCG: q; RES: x_new
    RI* rout;           // RES: r (inner precision)
    R* bout;            // APPLY: optional b
    const R* rhs_vec;   // RES: rhs vector instead of the frame load (adjoint), or null
    int first;          // RES: first residual of a solve (no correction, ||b|| formed)
    double rtol, inner_rtol, pass_frac;
    int max_inner;
    int* err;           // device error word (index checks of the bounds-check build)
};

template <typename R, typename C, typename RI, int MODE, bool WANT_B, int NW, typename T = R, bool ELD = false,
          bool LAM = true>
__global__ void __launch_bounds__(NW * 32) k_apply(const ApplyParams<R, C, RI> P) {
    // R: storage type of in/out (and of the PCG scalars); T: arithmetic of
    // the element contributions (R itself, or double-float for the residual
    // of the FP32 path); ELD: element data from the K_rho planes instead of
    // the frames; LAM: a per-element lambda may be set (false: the constant
    // lambda only, without the registers of that branch)
    constexpr int NT = NW * 32;
    __shared__ double sh_red[NT / 32];
    __shared__ int sh_last;
    const int4 bi = P.blocks[blockIdx.x];
    const int pair = bi.x;
    const PairDesc pd = P.pairs[pair];
    const int W = pd.W, H = pd.H, pitch = pd.pitch;
    const long long plane = (long long)H * pitch;

    R beta = R(0);
    R a_prev = R(0);
    int it = 0;
    bool corr = false;  // RES: fold the inner correction d + a p into x
    bool pcg_first = false;  // PCG: first iteration of a pass (p = z, d = 0)
    if (MODE == MODE_PCG) {
        if (P.sc_in[pair].done) return;  // uniform over the pair's blocks
        beta = (R)P.sc_in[pair].beta;
        a_prev = (R)P.sc_in[pair].a;
        it = P.sc_in[pair].it;
        pcg_first = (it == 0);
    }
    if (MODE == MODE_RES) {
        it = P.sc_in[pair].it;
        corr = !P.first && it > 0;
        a_prev = corr ? (R)P.sc_in[pair].a : R(0);
    }
    constexpr bool IS_RES = (MODE == MODE_RES) || (MODE == MODE_RESB);
    DF a_df = DF{0.f, 0.f};
    if constexpr (MODE == MODE_RES && std::is_same<T, DF>::value) a_df = Cvt<DF>::from((double)a_prev);

    const C* f1 = P.f1 + pd.frame_off;
    const C* f2 = P.f2 + pd.frame_off;
    const C* al = P.alpha + 2 * pd.frame_off;
    const long long vo = pd.vec_off;
    const R* vin = P.in + vo;
    const RI* pold = nullptr;
    RI* pnew = nullptr;
    if (MODE == MODE_PCG) {
        pold = ((it & 1) ? P.p_buf1 : P.p_buf0) + vo;
        pnew = ((it & 1) ? P.p_buf0 : P.p_buf1) + vo;
    }
    if (MODE == MODE_RES) pold = ((it & 1) ? P.p_buf1 : P.p_buf0) + vo;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int X0 = bi.y * (31 * NW);
    const int cx = X0 + 31 * warp - 1 + lane;  // square column / load column of this lane
    const int Y0 = bi.z * P.rows_per_block;
    const int Y1 = min(Y0 + P.rows_per_block, H);
    const bool mycol_owned = (lane >= 1) && (cx < W) && (cx >= 0);  // side-effect writes
    const bool out_col = (lane < 31) && (cx + 1 < W);
    const T lam = Cvt<T>::from(P.lam);
    const T gms = Cvt<T>::from(P.gms);
    constexpr T zero = kconst<T>(0.0);

    // load node (x, y) of the input vector + frames, with the mode's fused
    // update; side effects (p_new, d, x_new) only for owned nodes
    auto load = [&](int x, int y, bool owner) -> NodeVal<T> {
        NodeVal<T> v;
        const bool in = (x >= 0) && (x < W) && (y >= 0) && (y < H) &&
                        OF_CHECK(P.err, (long long)y * pitch + x, plane);
        if (!in) { v.p = v3(zero, zero, zero); v.f1 = zero; v.f2 = zero; return v; }
        const long long o = (long long)y * pitch + x;
        if constexpr (ELD) {
            v.f1 = zero; v.f2 = zero;
        } else {
            v.f1 = Cvt<T>::from(f1[o]);
            v.f2 = Cvt<T>::from(f2[o]);
        }
        if (MODE == MODE_RESB) {
            v.p = v3(zero, zero, zero);
            return v;
        }
        R p0 = vin[o], p1 = vin[o + plane], p2 = vin[o + 2 * plane];
        if constexpr (MODE == MODE_RES && std::is_same<T, DF>::value) {
            // FP32 path: x + (d + a p) in double-float on the FP32 pipe, stored as FP64
            DF X[3] = {Cvt<DF>::from(p0), Cvt<DF>::from(p1), Cvt<DF>::from(p2)};
            if (corr) {
                const RI* d = P.dcorr + vo;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const long long oc = o + c * plane;
                    X[c] = X[c] + (DF{(float)d[oc], 0.f} + a_df * DF{(float)pold[oc], 0.f});
                }
            }
            if (owner && P.out) {
                R* xn = P.out + vo;
#pragma unroll
                for (int c = 0; c < 3; ++c) xn[o + c * plane] = df_to_double_bits(X[c]);
            }
            v.p = v3(X[0], X[1], X[2]);
            return v;
        }
        if (MODE == MODE_PCG) {
            if (!pcg_first) {
                R q0 = pold[o], q1 = pold[o + plane], q2 = pold[o + 2 * plane];
                if (owner) {
                    RI* d = P.dcorr + vo;
                    d[o] += (RI)(a_prev * q0);
                    d[o + plane] += (RI)(a_prev * q1);
                    d[o + 2 * plane] += (RI)(a_prev * q2);
                }
                p0 = p0 + beta * q0; p1 = p1 + beta * q1; p2 = p2 + beta * q2;
            } else if (owner) {
                RI* d = P.dcorr + vo;
                d[o] = RI(0); d[o + plane] = RI(0); d[o + 2 * plane] = RI(0);
            }
            if (owner) { pnew[o] = p0; pnew[o + plane] = p1; pnew[o + 2 * plane] = p2; }
        }
        if (MODE == MODE_RES) {
            if (corr) {
                const RI* d = P.dcorr + vo;
                p0 = p0 + ((R)d[o] + a_prev * (R)pold[o]);
                p1 = p1 + ((R)d[o + plane] + a_prev * (R)pold[o + plane]);
                p2 = p2 + ((R)d[o + 2 * plane] + a_prev * (R)pold[o + 2 * plane]);
            }
            if (owner && P.out) {
                R* xn = P.out + vo;
                xn[o] = p0; xn[o + plane] = p1; xn[o + 2 * plane] = p2;
            }
        }
        v.p = v3(Cvt<T>::from(p0), Cvt<T>::from(p1), Cvt<T>::from(p2));
        return v;
    };
    auto shfl_node = [&](const NodeVal<T>& v) -> NodeVal<T> {
        NodeVal<T> w;
        w.p = shfl_down3(v.p);
        if constexpr (ELD) {
            w.f1 = v.f1; w.f2 = v.f2;
        } else {
            w.f1 = shfl_down(v.f1, 1);
            w.f2 = shfl_down(v.f2, 1);
        }
        return w;
    };

    R acc = R(0);          // PCG: per-thread partial of p.q (inner precision)
    T acc_r = zero, acc_b = zero;  // RES: per-thread ||r||^2, ||rhs||^2
    // prologue: node row Y0-1
    NodeVal<T> cur = load(cx, Y0 - 1, false);
    NodeVal<T> ncur = shfl_node(cur);
    if (lane == 31) ncur = load(cx + 1, Y0 - 1, false);
    V3<T> carry = v3(zero, zero, zero), carry_b = v3(zero, zero, zero);
    for (int sy = Y0 - 1; sy < Y1; ++sy) {
        const bool row_owned = (sy + 1 >= Y0) && (sy + 1 < Y1);
        // lane 31 also loads the node right of its column (no lane holds it);
        // one copy of the load's code serves both (a smaller loop body)
        NodeVal<T> nxt, nnxt;
#pragma unroll 1
        for (int k = 0; k < (lane == 31 ? 2 : 1); ++k) {
            const NodeVal<T> v = load(cx + k, sy + 1, k == 0 && mycol_owned && row_owned);
            if (k == 0) nxt = v;
            else nnxt = v;
        }
        {
            const NodeVal<T> sh = shfl_node(nxt);
            if (lane != 31) nnxt = sh;
        }
        const bool valid = (cx >= 0) && (cx < W - 1) && (sy >= 0) && (sy < H - 1);
        const T al0 = valid ? Cvt<T>::from(al[2 * ((long long)sy * pitch + cx)]) : zero;
        const T al1 = valid ? Cvt<T>::from(al[2 * ((long long)sy * pitch + cx) + 1]) : zero;
        V3<T> cA, cB, cC, cD, bA, bB, bC, bD;
        if constexpr (ELD) {
            T e0[9], e1[9];
            const C* ep = P.eld + pd.frame_off + (long long)sy * pitch + cx;
            constexpr int NK = (WANT_B || IS_RES) ? 9 : 6;  // F only for the load
            constexpr int K0 = (MODE == MODE_RESB) ? 6 : 0;  // A not needed for r = b
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const bool need = valid && k >= K0 && k < NK;
                e0[k] = need ? Cvt<T>::from(ep[k * P.eld_stride]) : zero;
                e1[k] = need ? Cvt<T>::from(ep[(9 + k) * P.eld_stride]) : zero;
            }
            square_contrib_el<T, WANT_B || IS_RES, MODE != MODE_RESB>(cur.p, ncur.p, nnxt.p, nxt.p, al0, al1, lam, e0,
                                                                      e1, valid, cA, cB, cC, cD, bA, bB, bC, bD);
        } else if (LAM && P.lamel) {
            const C* la = P.lamel + 2 * pd.frame_off;
            const T la0 = valid ? Cvt<T>::from(la[2 * ((long long)sy * pitch + cx)]) : zero;
            const T la1 = valid ? Cvt<T>::from(la[2 * ((long long)sy * pitch + cx) + 1]) : zero;
            square_contrib_l<T, WANT_B || IS_RES, MODE != MODE_RESB>(cur, ncur, nnxt, nxt, al0, al1, la0, la1, gms,
                                                                        valid, cA, cB, cC, cD, bA, bB, bC, bD);
        } else {
            square_contrib<T, WANT_B || IS_RES, MODE != MODE_RESB>(cur, ncur, nnxt, nxt, al0, al1, lam, gms, valid,
                                                                      cA, cB, cC, cD, bA, bB, bC, bD);
        }
        V3<T> left = shfl_down3(cA);
        V3<T> res = carry + cB + left;  // node (cx+1, sy) complete
        V3<T> resb = v3(zero, zero, zero);
        constexpr bool NEED_B = WANT_B || IS_RES;
        if constexpr (NEED_B) resb = carry_b + bB + shfl_down3(bA);
        if (sy >= Y0 && out_col && OF_CHECK(P.err, (long long)sy * pitch + (cx + 1), plane)) {
            const long long o = (long long)sy * pitch + (cx + 1);
            if constexpr (MODE == MODE_APPLY || MODE == MODE_PCG) {
                R* q = P.out + vo;
                q[o] = res.a; q[o + plane] = res.b; q[o + 2 * plane] = res.c;
                if constexpr (MODE == MODE_PCG) acc += ncur.p.a * res.a + ncur.p.b * res.b + ncur.p.c * res.c;
                if constexpr (WANT_B) {
                    if (P.bout) {
                        R* bo = P.bout + vo;
                        bo[o] = resb.a; bo[o + plane] = resb.b; bo[o + 2 * plane] = resb.c;
                    }
                }
            }
            if constexpr (IS_RES) {
                V3<T> rhs;
                if (P.rhs_vec) {
                    const R* c = P.rhs_vec + vo;
                    rhs = v3(Cvt<T>::from(c[o]), Cvt<T>::from(c[o + plane]), Cvt<T>::from(c[o + 2 * plane]));
                } else {
                    rhs = resb;
                }
                V3<T> r = v3(rhs.a - res.a, rhs.b - res.b, rhs.c - res.c);
                RI* ro = P.rout + vo;
                ro[o] = Cvt<RI>::from(r.a); ro[o + plane] = Cvt<RI>::from(r.b); ro[o + 2 * plane] = Cvt<RI>::from(r.c);
                acc_r = acc_r + (r.a * r.a + r.b * r.b + r.c * r.c);
                acc_b = acc_b + (rhs.a * rhs.a + rhs.b * rhs.b + rhs.c * rhs.c);
            }
        }
        carry = cC + shfl_down3(cD);
        if constexpr (NEED_B) carry_b = bC + shfl_down3(bD);
        cur = nxt;
        ncur = nnxt;
    }

    if constexpr (MODE == MODE_APPLY) return;
    // ---- block partials and last-block reduction of the pair
    double s0, s1 = 0.0;
    if constexpr (MODE == MODE_PCG) {
        s0 = block_sum<NT>((double)acc, sh_red);
    } else if constexpr (std::is_same<T, DF>::value) {
        // double-float block sums (the FP64 pipe is narrow), one conversion
        const DF r2 = df_block_sum<NT>(acc_r, reinterpret_cast<DF*>(sh_red));
        const DF b2 = df_block_sum<NT>(acc_b, reinterpret_cast<DF*>(sh_red));
        s0 = threadIdx.x == 0 ? df_to_double(r2) : 0.0;
        s1 = threadIdx.x == 0 ? df_to_double(b2) : 0.0;
    } else {
        s0 = block_sum<NT>(Cvt<double>::from(acc_r), sh_red);
        s1 = block_sum<NT>(Cvt<double>::from(acc_b), sh_red);
    }
    if (threadIdx.x == 0) {
        P.partial[2 * (long long)bi.w] = s0;
        P.partial[2 * (long long)bi.w + 1] = s1;
    }
    if (!arrive_last(&P.counter[pair], (unsigned)pd.nblk, &sh_last)) return;
    double t0 = ordered_sum<NT>(P.partial + 2 * (long long)pd.blk0, pd.nblk, 2, sh_red);
    double t1 = IS_RES ? ordered_sum<NT>(P.partial + 2 * (long long)pd.blk0 + 1, pd.nblk, 2, sh_red) : 0.0;
    if (threadIdx.x == 0) {
        PairScalars* s = P.sc + pair;
        if (MODE == MODE_PCG) {
            s->pq = t0;
            if (!(t0 > 0.0) || !isfinite(t0) || !isfinite(s->rz)) {
                s->a = 0.0;
                s->done = 1;
                s->status = 6;
            } else {
                s->a = s->rz / t0;
            }
        } else {  // MODE_RES: set up the inner pass
            s->res2 = t0;
            if (P.first || MODE == MODE_RESB) s->bnorm2 = t1;
            const double b2 = s->bnorm2;
            const bool conv = (t0 <= P.rtol * P.rtol * b2) || (t0 == 0.0);
            // the pass aims at pass_frac times the outer tolerance
            double rel = P.pass_frac * P.rtol * sqrt(b2 / (t0 > 0.0 ? t0 : 1.0));
            if (rel < P.inner_rtol) rel = P.inner_rtol;
            if (rel > 0.5) rel = 0.5;
            s->tol2 = rel * rel * t0;
            s->it = 0;
            s->done = conv ? 1 : 0;
            s->status = isfinite(t0) ? 0 : 6;
            if (!isfinite(t0)) s->done = 1;
            s->max_it = P.max_inner;
            s->a = 0.0;
            s->pad[0] = conv ? 1 : 0;  // outer convergence flag
        }
        __threadfence();
        P.counter[pair] = 0u;
    }
}

}  // namespace ofk

namespace ofk {

// FP32 apply with four columns per lane (PCG and APPLY modes).
//
// One warp per block covers 124 output columns x rows_per_block rows: lane l
// holds columns X0 - 4 + 4l .. X0 - 1 + 4l as float4 (lane 0's columns are a
// halo) and forms the two triangles of the four squares whose left corners
// are those columns.  The fourth square needs the next lane's first column
// (one shuffle of 5 values); the first node of a lane receives the right
// corners of the previous lane's last square (one shuffle of 2 x 3 values).
// Lane 31's last square needs column X0 + 124, fetched separately.  Every
// element is formed once; every word is read once per warp plus a 4-column
// halo and the row above the block.
//
// Rows stream through a per-warp ring of three shared-memory stages filled
// with cp.async (16-byte LDGSTS, zero-filled outside the image): while node
// row y is combined with row y-1, row y+1 is already in flight, without
// holding those loads in registers.
struct Node4 {
    float4 p0, p1, p2, f1, f2;
};

__device__ __forceinline__ NodeVal<float> pick(const Node4& n, int j) {
    NodeVal<float> v;
    const float* a = reinterpret_cast<const float*>(&n.p0);
    const float* b = reinterpret_cast<const float*>(&n.p1);
    const float* c = reinterpret_cast<const float*>(&n.p2);
    const float* d = reinterpret_cast<const float*>(&n.f1);
    const float* e = reinterpret_cast<const float*>(&n.f2);
    v.p = v3(a[j], b[j], c[j]);
    v.f1 = d[j];
    v.f2 = e[j];
    return v;
}

__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }
__device__ __forceinline__ float4 fma4(float s, float4 x, float4 y) {
    return make_float4(fmaf(s, x.x, y.x), fmaf(s, x.y, y.y), fmaf(s, x.z, y.z), fmaf(s, x.w, y.w));
}
__device__ __forceinline__ float4 mask4(float4 v, int c0, int W) {
    // zero the columns at or beyond W (pitch padding)
    if (c0 + 0 >= W) v.x = 0.f;
    if (c0 + 1 >= W) v.y = 0.f;
    if (c0 + 2 >= W) v.z = 0.f;
    if (c0 + 3 >= W) v.w = 0.f;
    return v;
}

// cp.async with a source size of 0 writes zeros and reads nothing
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

constexpr int A4_NS = 3;     // ring stages
constexpr int A4_NARR = 13;  // float4 slots per lane, row and stage
enum { A4_F1, A4_F2, A4_Z0, A4_Z1, A4_Z2, A4_Q0, A4_Q1, A4_Q2, A4_D0, A4_D1, A4_D2, A4_AL0, A4_AL1 };
constexpr int A4_EXTRA = 8;  // floats of column X0 + 124 per stage: f1, f2, z0..z2, q0..q2
__host__ __device__ constexpr int apply4_smem_bytes() { return A4_NS * (A4_NARR * 32 * 16 + A4_EXTRA * 4); }

template <int MODE>
__global__ void __launch_bounds__(32, 16) k_apply4(const ApplyParams<float, float, float> P) {
    extern __shared__ float4 a4_ring[];
    const int4 bi = P.blocks[blockIdx.x];
    const int pair = bi.x;
    const PairDesc pd = P.pairs[pair];
    const int W = pd.W, H = pd.H, pitch = pd.pitch;
    const long long plane = (long long)H * pitch;
    float beta = 0.f, a_prev = 0.f;
    int it = 0;
    bool first = false;
    if (MODE == MODE_PCG) {
        if (P.sc_in[pair].done) return;
        beta = f32_from_double(P.sc_in[pair].beta);  // integer conversions: the FP64 pipe is narrow
        a_prev = f32_from_double(P.sc_in[pair].a);
        it = P.sc_in[pair].it;
        first = (it == 0);
    }
    const bool use_q = (MODE == MODE_PCG) && !first;  // p = z + beta p_old, d += a_prev p_old
    const float* f1 = P.f1 + pd.frame_off;
    const float* f2 = P.f2 + pd.frame_off;
    const float* al = P.alpha + 2 * pd.frame_off;
    const long long vo = pd.vec_off;
    const float* vin = P.in + vo;
    const float* pold = vin;
    float* pnew = nullptr;
    float* dcor = nullptr;
    if (MODE == MODE_PCG) {
        pold = ((it & 1) ? P.p_buf1 : P.p_buf0) + vo;
        pnew = ((it & 1) ? P.p_buf0 : P.p_buf1) + vo;
        dcor = P.dcorr + vo;
    }
    const int lane = threadIdx.x;
    const int X0 = bi.y * 124;
    const int c0 = X0 - 4 + 4 * lane;      // first of this lane's four columns
    const int Y0 = bi.z * P.rows_per_block;
    const int Y1 = min(Y0 + P.rows_per_block, H);
    const int nrows = Y1 - Y0 + 2;         // node rows Y0 - 1 .. Y1
    const bool own = lane >= 1 && c0 < W;  // this lane's columns are output columns
    const float lam = P.lam, gms = P.gms;
    float* extra = reinterpret_cast<float*>(a4_ring + A4_NS * A4_NARR * 32);

    auto slot = [&](int s, int a) -> float4* { return a4_ring + (s * A4_NARR + a) * 32 + lane; };
    // node row j (y = Y0 - 1 + j) and square row y of alpha into stage j mod 3
    auto issue = [&](int j) {
        const int s = j % A4_NS, y = Y0 - 1 + j;
        const bool rv = y >= 0 && y < H && c0 >= 0 && c0 < W && OF_CHECK(P.err, (long long)y * pitch + c0 + 3, plane);
        const long long o = rv ? (long long)y * pitch + c0 : 0;
        cp_async16(slot(s, A4_F1), f1 + o, rv);
        cp_async16(slot(s, A4_F2), f2 + o, rv);
        cp_async16(slot(s, A4_Z0), vin + o, rv);
        cp_async16(slot(s, A4_Z1), vin + o + plane, rv);
        cp_async16(slot(s, A4_Z2), vin + o + 2 * plane, rv);
        if (use_q) {
            cp_async16(slot(s, A4_Q0), pold + o, rv);
            cp_async16(slot(s, A4_Q1), pold + o + plane, rv);
            cp_async16(slot(s, A4_Q2), pold + o + 2 * plane, rv);
            if (own && y >= Y0 && y < Y1) {
                cp_async16(slot(s, A4_D0), dcor + o, true);
                cp_async16(slot(s, A4_D1), dcor + o + plane, true);
                cp_async16(slot(s, A4_D2), dcor + o + 2 * plane, true);
            }
        }
        if (j < nrows - 1) {  // square row y is used
            const bool av = y >= 0 && y < H - 1 && c0 >= 0 && c0 < W - 1 &&
                            OF_CHECK(P.err, 2 * ((long long)y * pitch + c0) + 7, 2 * plane);
            const long long oa = av ? 2 * ((long long)y * pitch + c0) : 0;
            cp_async16(slot(s, A4_AL0), al + oa, av);
            cp_async16(slot(s, A4_AL1), al + oa + 4, av);
        }
        if (lane == 31) {
            const int x = c0 + 4;
            const bool ev = y >= 0 && y < H && x < W && OF_CHECK(P.err, (long long)y * pitch + x, plane);
            const long long oe = ev ? (long long)y * pitch + x : 0;
            float* e = extra + s * A4_EXTRA;
            cp_async4(e + 0, f1 + oe, ev);
            cp_async4(e + 1, f2 + oe, ev);
            cp_async4(e + 2, vin + oe, ev);
            cp_async4(e + 3, vin + oe + plane, ev);
            cp_async4(e + 4, vin + oe + 2 * plane, ev);
            if (use_q) {
                cp_async4(e + 5, pold + oe, ev);
                cp_async4(e + 6, pold + oe + plane, ev);
                cp_async4(e + 7, pold + oe + 2 * plane, ev);
            }
        }
    };
    // node row j from its stage, with the fused PCG updates (owned rows)
    auto finish = [&](int j) -> Node4 {
        const int s = j % A4_NS, y = Y0 - 1 + j;
        Node4 n;
        n.f1 = mask4(*slot(s, A4_F1), c0, W);
        n.f2 = mask4(*slot(s, A4_F2), c0, W);
        float4 a = *slot(s, A4_Z0), b = *slot(s, A4_Z1), c = *slot(s, A4_Z2);
        float4 qa = f4(0.f), qb = f4(0.f), qc = f4(0.f);
        if (use_q) {
            qa = *slot(s, A4_Q0);
            qb = *slot(s, A4_Q1);
            qc = *slot(s, A4_Q2);
            a = fma4(beta, qa, a);
            b = fma4(beta, qb, b);
            c = fma4(beta, qc, c);
        }
        // pitch padding of p_new is written as zeros
        a = mask4(a, c0, W);
        b = mask4(b, c0, W);
        c = mask4(c, c0, W);
        if (MODE == MODE_PCG && own && y >= Y0 && y < Y1 && OF_CHECK(P.err, (long long)y * pitch + c0 + 3, plane)) {
            const long long o = (long long)y * pitch + c0;
            if (use_q) {
                *reinterpret_cast<float4*>(dcor + o) = fma4(a_prev, qa, *slot(s, A4_D0));
                *reinterpret_cast<float4*>(dcor + o + plane) = fma4(a_prev, qb, *slot(s, A4_D1));
                *reinterpret_cast<float4*>(dcor + o + 2 * plane) = fma4(a_prev, qc, *slot(s, A4_D2));
            } else {
                *reinterpret_cast<float4*>(dcor + o) = f4(0.f);
                *reinterpret_cast<float4*>(dcor + o + plane) = f4(0.f);
                *reinterpret_cast<float4*>(dcor + o + 2 * plane) = f4(0.f);
            }
            *reinterpret_cast<float4*>(pnew + o) = a;
            *reinterpret_cast<float4*>(pnew + o + plane) = b;
            *reinterpret_cast<float4*>(pnew + o + 2 * plane) = c;
        }
        n.p0 = a;
        n.p1 = b;
        n.p2 = c;
        return n;
    };
    // first column of the next lane (lane 31: column X0 + 124 from its slot)
    auto right = [&](const Node4& n, int j) -> NodeVal<float> {
        NodeVal<float> v;
        v.p = v3(__shfl_down_sync(0xffffffffu, n.p0.x, 1), __shfl_down_sync(0xffffffffu, n.p1.x, 1),
                 __shfl_down_sync(0xffffffffu, n.p2.x, 1));
        v.f1 = __shfl_down_sync(0xffffffffu, n.f1.x, 1);
        v.f2 = __shfl_down_sync(0xffffffffu, n.f2.x, 1);
        if (lane == 31) {
            const float* e = extra + (j % A4_NS) * A4_EXTRA;
            float p0 = e[2], p1 = e[3], p2 = e[4];
            if (use_q) {
                p0 = fmaf(beta, e[5], p0);
                p1 = fmaf(beta, e[6], p1);
                p2 = fmaf(beta, e[7], p2);
            }
            v.p = v3(p0, p1, p2);
            v.f1 = e[0];
            v.f2 = e[1];
        }
        return v;
    };

    float acc = 0.f;
    V3<float> carry[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) carry[j] = v3(0.f, 0.f, 0.f);
    Node4 cur;
    NodeVal<float> rcur;
    issue(0);
    cp_async_commit();
    for (int j = 0; j < nrows; ++j) {
        if (j + 1 < nrows) issue(j + 1);
        cp_async_commit();  // one group per row (possibly empty): row j is the older one
        cp_async_wait1();
        const Node4 nxt = finish(j);
        const NodeVal<float> rnxt = right(nxt, j);
        if (j >= 1) {
            // square row sy between node rows sy (cur) and sy + 1 (nxt)
            const int sy = Y0 - 2 + j;
            const bool rowv = (sy >= 0) && (sy < H - 1) && c0 >= 0 && c0 < W - 1;
            const float4 alA = *slot((j - 1) % A4_NS, A4_AL0), alB = *slot((j - 1) % A4_NS, A4_AL1);
            const float alv[8] = {alA.x, alA.y, alA.z, alA.w, alB.x, alB.y, alB.z, alB.w};
            V3<float> cA[4], cB[4], cC[4], cD[4], bdum;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool valid = rowv && (c0 + k < W - 1);
                const NodeVal<float> A = pick(cur, k), D = pick(nxt, k);
                const NodeVal<float> B = (k < 3) ? pick(cur, k + 1) : rcur;
                const NodeVal<float> C = (k < 3) ? pick(nxt, k + 1) : rnxt;
                square_contrib<float, false>(A, B, C, D, alv[2 * k], alv[2 * k + 1], lam, gms, valid, cA[k], cB[k],
                                             cC[k], cD[k], bdum, bdum, bdum, bdum);
            }
            // right corners of the previous lane's last square
            const V3<float> pB = v3(__shfl_up_sync(0xffffffffu, cB[3].a, 1), __shfl_up_sync(0xffffffffu, cB[3].b, 1),
                                    __shfl_up_sync(0xffffffffu, cB[3].c, 1));
            const V3<float> pC = v3(__shfl_up_sync(0xffffffffu, cC[3].a, 1), __shfl_up_sync(0xffffffffu, cC[3].b, 1),
                                    __shfl_up_sync(0xffffffffu, cC[3].c, 1));
            V3<float> out[4];
            out[0] = carry[0] + cA[0] + pB;
#pragma unroll
            for (int k = 1; k < 4; ++k) out[k] = carry[k] + cA[k] + cB[k - 1];
            if (sy >= Y0 && own && OF_CHECK(P.err, (long long)sy * pitch + c0 + 3, plane)) {
                const long long o = (long long)sy * pitch + c0;
                float* q = P.out + vo;
                *reinterpret_cast<float4*>(q + o) = make_float4(out[0].a, out[1].a, out[2].a, out[3].a);
                *reinterpret_cast<float4*>(q + o + plane) = make_float4(out[0].b, out[1].b, out[2].b, out[3].b);
                *reinterpret_cast<float4*>(q + o + 2 * plane) = make_float4(out[0].c, out[1].c, out[2].c, out[3].c);
                if (MODE == MODE_PCG) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const NodeVal<float> pk = pick(cur, k);
                        acc += pk.p.a * out[k].a + pk.p.b * out[k].b + pk.p.c * out[k].c;
                    }
                }
            }
            carry[0] = cD[0] + pC;
#pragma unroll
            for (int k = 1; k < 4; ++k) carry[k] = cD[k] + cC[k - 1];
        }
        cur = nxt;
        rcur = rnxt;
    }
    if (MODE == MODE_APPLY) return;
    // p.q in two levels, so that no block reads more than one partial per
    // lane and round: the warp partial (FP32 within the warp) goes to the
    // block's slot; the last block of each group of 32 consecutive blocks sums
    // the group's partials in order into the group slot (the odd slot of the
    // group's first block); the pair's last group sums the group slots in
    // order (double-float arithmetic throughout)
    const float s0 = warp_sum(acc);
    if (P.pq_fixed) {
        // one pair: the fixed-point sum (no arrival, no serial tail; see pq_fix_shift)
        if (lane == 0) {
            PairScalars* sp = P.sc + pair;
            const int k = pq_fix_shift(P.sc_in[pair].rz);
            const float v = __fmul_rn(s0, __int_as_float((127 + k) << 23));  // exact: a power of two
            // 2^62 (false for NaN and infinities); the sum overflows only if the
            // partials' magnitudes add up to 2^23 |r.z| (a < 1e-7), reported
            // like a non-finite p.q: as a breakdown
            if (fabsf(v) < 4.611686e18f)
                atomicAdd(reinterpret_cast<unsigned long long*>(&sp->pq_fix), (unsigned long long)__float2ll_rn(v));
            else
                atomicOr(&sp->pad[1], 1);
        }
        return;
    }
    __shared__ int sh_last;
    if (lane == 0) P.partial[2 * (long long)bi.w] = (double)s0;
    const int g = (bi.w - pd.blk0) >> 5;
    const int gfirst = pd.blk0 + 32 * g, gsize = min(32, pd.nblk - 32 * g);
    if (!arrive_last(&P.gcounter[gfirst], (unsigned)gsize, &sh_last)) return;
    {
        const DF v = lane < gsize ? df_from_double(__ldcg(P.partial + 2 * (long long)(gfirst + lane))) : DF{0.f, 0.f};
        const DF sg = df_warp_sum(v);
        if (lane == 0) {
            P.partial[2 * (long long)gfirst + 1] = df_to_double(sg);
            P.gcounter[gfirst] = 0u;
        }
    }
    const int ngroups = (pd.nblk + 31) >> 5;
    if (!arrive_last(&P.counter[pair], (unsigned)ngroups, &sh_last)) return;
    PairScalars* s = P.sc + pair;
    const double rz = s->rz;  // loaded alongside the group slots
    const DF t0d = df_warp_sum(df_strided_sum<8>(P.partial + 2 * (long long)pd.blk0 + 1, ngroups, 64, lane, 32));
    if (lane == 0) {
        const double t0 = df_to_double(t0d);
        s->pq = t0;
        if (!(t0 > 0.0) || !isfinite(t0) || !isfinite(rz)) {
            s->a = 0.0;
            s->done = 1;
            s->status = 6;
        } else {
            s->a = rz / t0;
        }
        P.counter[pair] = 0u;
    }
}

}  // namespace ofk
