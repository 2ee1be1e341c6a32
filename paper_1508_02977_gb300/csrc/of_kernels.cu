// Kernel instantiations and launchers of the solve path.
#include "of_apply.cuh"
#include "of_launch.h"
#include "of_schwarz.cuh"

namespace ofl {

using namespace ofk;

static constexpr int APPLY_NW = 4;    // warps per apply block (124 output columns)
static constexpr int SCHWARZ_NT = 256;

// ------------------------------------------------------------ copy2d --
template <typename S, typename D>
__global__ void k_copy2d(const S* __restrict__ src, long long sp, D* __restrict__ dst, long long dp, long long rows,
                         long long cols) {
    const long long n = rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / cols, c = i - r * cols;
        dst[r * dp + c] = (D)src[r * sp + c];
    }
}
template <typename D>
__global__ void k_fill2d(D* dst, long long dp, long long rows, long long cols, D v) {
    const long long n = rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / cols, c = i - r * cols;
        dst[r * dp + c] = v;
    }
}

static unsigned grid_for(long long n, int nt) {
    long long g = (n + nt - 1) / nt;
    if (g > 152LL * 64) g = 152LL * 64;
    if (g < 1) g = 1;
    return (unsigned)g;
}

cudaError_t copy2d(const void* src, int stype, long long spitch, void* dst, int dtype, long long dpitch,
                   long long rows, long long cols, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const unsigned g = grid_for(rows * cols, 256);
    if (stype == T_F32 && dtype == T_F32)
        k_copy2d<float, float><<<g, 256, 0, st>>>((const float*)src, spitch, (float*)dst, dpitch, rows, cols);
    else if (stype == T_F32 && dtype == T_F64)
        k_copy2d<float, double><<<g, 256, 0, st>>>((const float*)src, spitch, (double*)dst, dpitch, rows, cols);
    else if (stype == T_F64 && dtype == T_F32)
        k_copy2d<double, float><<<g, 256, 0, st>>>((const double*)src, spitch, (float*)dst, dpitch, rows, cols);
    else
        k_copy2d<double, double><<<g, 256, 0, st>>>((const double*)src, spitch, (double*)dst, dpitch, rows, cols);
    return cudaGetLastError();
}

cudaError_t fill2d(void* dst, int dtype, long long dpitch, long long rows, long long cols, double v, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const unsigned g = grid_for(rows * cols, 256);
    if (dtype == T_F32) k_fill2d<float><<<g, 256, 0, st>>>((float*)dst, dpitch, rows, cols, (float)v);
    else k_fill2d<double><<<g, 256, 0, st>>>((double*)dst, dpitch, rows, cols, v);
    return cudaGetLastError();
}

// ------------------------------------------------------------- solve --
template <typename R, typename C, typename RI>
static ApplyParams<R, C, RI> base_params(const SolveBufs& B) {
    ApplyParams<R, C, RI> P;
    memset(&P, 0, sizeof(P));
    P.pairs = B.pairs;
    P.blocks = B.blocks;
    P.sc_in = B.sc;
    P.sc = B.sc;
    P.partial = B.partA;
    P.counter = B.cntA;
    P.f1 = (const C*)B.f1;
    P.f2 = (const C*)B.f2;
    P.alpha = (const C*)B.alpha;
    P.lam = (R)B.lam;
    P.rows_per_block = B.rows_per_block;
    return P;
}

template <typename C, typename RI>
static cudaError_t residual_t(const SolveBufs& B, const double* xin, double* xout, const double* rhs_vec, int first,
                              double rtol, double inner_rtol, int max_inner, cudaStream_t st) {
    auto P = base_params<double, C, RI>(B);
    P.in = xin;
    P.p_buf0 = (RI*)B.p0;
    P.p_buf1 = (RI*)B.p1;
    P.dcorr = (RI*)B.d;
    P.out = xout;
    P.rout = (RI*)B.r;
    P.rhs_vec = rhs_vec;
    P.first = first;
    P.rtol = rtol;
    P.inner_rtol = inner_rtol;
    P.max_inner = max_inner;
    k_apply<double, C, RI, MODE_RES, false, APPLY_NW><<<B.nblk, APPLY_NW * 32, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_residual(const SolveBufs& B, const double* xin, double* xout, const double* rhs_vec, int first,
                            double rtol, double inner_rtol, int max_inner, cudaStream_t st) {
    if (B.fp64) return residual_t<double, double>(B, xin, xout, rhs_vec, first, rtol, inner_rtol, max_inner, st);
    return residual_t<float, float>(B, xin, xout, rhs_vec, first, rtol, inner_rtol, max_inner, st);
}

static SchwarzParams schwarz_params(const SolveBufs& B) {
    SchwarzParams S;
    memset(&S, 0, sizeof(S));
    S.pairs = B.pairs;
    S.tiles = B.tiles;
    S.tmaps = B.tmaps;
    S.sc = B.sc;
    S.partial = B.partS;
    S.counter = B.cntS;
    S.err = B.err;
    S.r = B.r;
    S.z = B.z;
    S.lam = B.lam;
    S.Tx = B.Tx;
    S.Ty = B.Ty;
    S.ov = B.ov;
    S.sweeps = B.sweeps;
    S.spin_limit = B.spin_limit;
    return S;
}

size_t schwarz_smem_bytes(int fp64, int Tx, int Ty, int ov) {
    return fp64 ? sch_smem_bytes<double>(Tx, Ty, ov) : sch_smem_bytes<float>(Tx, Ty, ov);
}

cudaError_t schwarz_configure(int fp64, size_t smem) {
    if (fp64)
        return cudaFuncSetAttribute(k_schwarz<double, SCHWARZ_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaFuncSetAttribute(k_schwarz<float, SCHWARZ_NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

static cudaError_t schwarz_launch(const SolveBufs& B, const SchwarzParams& S, int ntiles, cudaStream_t st) {
    const size_t smem = schwarz_smem_bytes(B.fp64, B.Tx, B.Ty, B.ov);
    if (B.fp64) k_schwarz<double, SCHWARZ_NT><<<ntiles, SCHWARZ_NT, smem, st>>>(S);
    else k_schwarz<float, SCHWARZ_NT><<<ntiles, SCHWARZ_NT, smem, st>>>(S);
    return cudaGetLastError();
}

cudaError_t launch_precond_first(const SolveBufs& B, cudaStream_t st) {
    SchwarzParams S = schwarz_params(B);
    S.first = 1;
    return schwarz_launch(B, S, B.ntiles, st);
}

template <typename R>
static cudaError_t pcg_apply_t(const SolveBufs& B, int first, cudaStream_t st) {
    auto P = base_params<R, R, R>(B);
    P.in = (const R*)B.z;
    P.p_buf0 = (R*)B.p0;
    P.p_buf1 = (R*)B.p1;
    P.dcorr = (R*)B.d;
    P.out = (R*)B.q;
    P.first = first;
    k_apply<R, R, R, MODE_PCG, false, APPLY_NW><<<B.nblk, APPLY_NW * 32, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_pcg_apply(const SolveBufs& B, int first, cudaStream_t st) {
    return B.fp64 ? pcg_apply_t<double>(B, first, st) : pcg_apply_t<float>(B, first, st);
}

cudaError_t launch_pcg_precond(const SolveBufs& B, cudaStream_t st) {
    SchwarzParams S = schwarz_params(B);
    return schwarz_launch(B, S, B.ntiles, st);
}

template <typename R>
static cudaError_t apply_t(const SolveBufs& B, int blk0, int nblk, const void* p, void* q, void* b, cudaStream_t st) {
    auto P = base_params<R, R, R>(B);
    P.blocks = B.blocks + blk0;
    P.in = (const R*)p;
    P.out = (R*)q;
    P.bout = (R*)b;
    if (b) k_apply<R, R, R, MODE_APPLY, true, APPLY_NW><<<nblk, APPLY_NW * 32, 0, st>>>(P);
    else k_apply<R, R, R, MODE_APPLY, false, APPLY_NW><<<nblk, APPLY_NW * 32, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_apply(const SolveBufs& B, int pair, int blk0, int nblk, const void* p, void* q, void* b,
                         cudaStream_t st) {
    (void)pair;
    return B.fp64 ? apply_t<double>(B, blk0, nblk, p, q, b, st) : apply_t<float>(B, blk0, nblk, p, q, b, st);
}

cudaError_t launch_precond_only(const SolveBufs& B, int tile0, int ntiles, cudaStream_t st) {
    SchwarzParams S = schwarz_params(B);
    S.tiles = B.tiles + tile0;
    S.apply_only = 1;
    S.first = 1;
    return schwarz_launch(B, S, ntiles, st);
}

}  // namespace ofl
