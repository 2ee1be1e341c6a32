// of_residual_noalloc: the FP64 residual b - A U of one frame pair for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a frame
// budget that forbids allocator calls (they can synchronise the device or
// fail under memory pressure), plug-ins whose host application owns every
// allocation, and code that must not touch an allocator between set-up and
// tear-down.  The handle-based entry points allocate their workspace in
// of_setup_grid, so they are closed to such callers.  This entry point needs
// no handle and allocates nothing: the caller passes the inputs and outputs,
// and the only scratch (one FP64 partial pair per thread block plus an
// arrival counter) is the file-scope array below, which every GPU that loads
// the library holds until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "of.h"
#include "of_apply.cuh"

namespace {

constexpr int NA_NW = 4;               // warps per block; 31 output columns per warp
constexpr int NA_COLS = 31 * NA_NW;    // 124 columns per block
constexpr int NA_ROWS = 32;            // rows per block
constexpr int NA_MAX_BLOCKS = 32768;   // scratch capacity (blocks of 124 x 32 nodes)
constexpr int NA_COUNTER = 2 * NA_MAX_BLOCKS;  // slot of the arrival counter
constexpr int NA_SCRATCH = 2 * NA_MAX_BLOCKS + 32;

// [2*b, 2*b+1]: ||r||^2 and ||b||^2 of block b; slot NA_COUNTER: arrival
// counter (its bits as an unsigned).  512 KB + 256 B per device.
static __device__ __align__(256) double g_noalloc_scratch[NA_SCRATCH];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mu;
// per device: the context the address was looked up in, and the address (a
// device reset destroys the context and the module with it: the address is
// then looked up again in the new context)
struct ScratchSlot {
    CUcontext ctx;
    double* ptr;
};
ScratchSlot g_slot[NA_MAX_DEVICES] = {};

// the calling thread's current context (driver entry point, no link to libcuda)
bool current_context(CUcontext* ctx) {
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return false;
        fn = (PFN_cuCtxGetCurrent_v4000)p;
    }
    return fn(ctx) == CUDA_SUCCESS;
}

// Column-streamed element apply in FP64 on the caller's layouts:
// frames [H][W], alpha [H-1][W-1][2], U and r [3][H][W].
__global__ void __launch_bounds__(NA_NW * 32)
    k_residual_noalloc(int W, int H, int nbx, const double* __restrict__ f1, const double* __restrict__ f2,
                       const double* __restrict__ alpha, double lam, const double* __restrict__ U,
                       double* __restrict__ r_out, double* __restrict__ norms_out, double* __restrict__ scratch) {
    using namespace ofk;
    __shared__ double sh_red[NA_NW];
    __shared__ int sh_last;
    const int bx = blockIdx.x % nbx, by = blockIdx.x / nbx;
    const long long plane = (long long)H * W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cx = bx * NA_COLS + 31 * warp - 1 + lane;
    const int Y0 = by * NA_ROWS, Y1 = min(Y0 + NA_ROWS, H);
    const bool out_col = (lane < 31) && (cx + 1 < W);
    auto load = [&](int x, int y) -> NodeVal<double> {
        NodeVal<double> v;
        if (x < 0 || x >= W || y < 0 || y >= H) {
            v.p = v3(0.0, 0.0, 0.0);
            v.f1 = v.f2 = 0.0;
            return v;
        }
        const long long o = (long long)y * W + x;
        v.f1 = f1[o];
        v.f2 = f2[o];
        v.p = v3(U[o], U[o + plane], U[o + 2 * plane]);
        return v;
    };
    auto shfl_node = [&](const NodeVal<double>& v) {
        NodeVal<double> w;
        w.p = shfl_down3(v.p);
        w.f1 = shfl_down(v.f1, 1);
        w.f2 = shfl_down(v.f2, 1);
        return w;
    };
    double acc_r = 0.0, acc_b = 0.0;
    NodeVal<double> cur = load(cx, Y0 - 1);
    NodeVal<double> ncur = shfl_node(cur);
    if (lane == 31) ncur = load(cx + 1, Y0 - 1);
    V3<double> carry = v3(0.0, 0.0, 0.0), carry_b = v3(0.0, 0.0, 0.0);
    for (int sy = Y0 - 1; sy < Y1; ++sy) {
        NodeVal<double> nxt = load(cx, sy + 1);
        NodeVal<double> nnxt = shfl_node(nxt);
        if (lane == 31) nnxt = load(cx + 1, sy + 1);
        const bool valid = (cx >= 0) && (cx < W - 1) && (sy >= 0) && (sy < H - 1);
        const long long ao = 2 * ((long long)sy * (W - 1) + cx);
        const double al0 = valid ? alpha[ao] : 0.0, al1 = valid ? alpha[ao + 1] : 0.0;
        V3<double> cA, cB, cC, cD, bA, bB, bC, bD;
        square_contrib<double, true>(cur, ncur, nnxt, nxt, al0, al1, lam, 1.0, valid, cA, cB, cC, cD, bA, bB, bC,
                                     bD);
        const V3<double> res = carry + cB + shfl_down3(cA);
        const V3<double> rhs = carry_b + bB + shfl_down3(bA);
        if (sy >= Y0 && out_col) {
            const long long o = (long long)sy * W + (cx + 1);
            const V3<double> r = v3(rhs.a - res.a, rhs.b - res.b, rhs.c - res.c);
            if (r_out) {
                r_out[o] = r.a;
                r_out[o + plane] = r.b;
                r_out[o + 2 * plane] = r.c;
            }
            acc_r += r.a * r.a + r.b * r.b + r.c * r.c;
            acc_b += rhs.a * rhs.a + rhs.b * rhs.b + rhs.c * rhs.c;
        }
        carry = cC + shfl_down3(cD);
        carry_b = bC + shfl_down3(bD);
        cur = nxt;
        ncur = nnxt;
    }
    const double s_r = block_sum<NA_NW * 32>(acc_r, sh_red);
    const double s_b = block_sum<NA_NW * 32>(acc_b, sh_red);
    if (threadIdx.x == 0) {
        scratch[2 * (long long)blockIdx.x] = s_r;
        scratch[2 * (long long)blockIdx.x + 1] = s_b;
    }
    unsigned* counter = reinterpret_cast<unsigned*>(scratch + NA_COUNTER);
    if (!arrive_last(counter, gridDim.x, &sh_last)) return;
    const double t_r = ordered_sum<NA_NW * 32>(scratch, gridDim.x, 2, sh_red);
    const double t_b = ordered_sum<NA_NW * 32>(scratch + 1, gridDim.x, 2, sh_red);
    if (threadIdx.x == 0) {
        norms_out[0] = t_b > 0.0 ? sqrt(t_r / t_b) : sqrt(t_r);
        norms_out[1] = t_r;
        norms_out[2] = t_b;
        __threadfence();
        *counter = 0u;
    }
}

}  // namespace

extern "C" of_status of_residual_noalloc(int W, int H, const double* f1, const double* f2, const double* alpha,
                                         double lambda, const double* U, double* r, double* norms, void* stream) {
    if (W < 2 || H < 2 || !f1 || !f2 || !alpha || !U || !norms || !(lambda > 0)) return OF_ERR_ARG;
    const int nbx = (W + NA_COLS - 1) / NA_COLS;
    const long long nblk = (long long)nbx * ((H + NA_ROWS - 1) / NA_ROWS);
    if (nblk > NA_MAX_BLOCKS) return OF_ERR_ARG;  // frame larger than the static scratch covers
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return OF_ERR_CUDA;
    double* scratch = nullptr;
    {
        // once per device (and again after a device reset), with that device
        // current: the device address of the scratch array (its host-side name
        // is only a stand-in).  cudaSetDevice makes the device's primary
        // context current in this thread, so that it can be compared.
        std::lock_guard<std::mutex> lk(g_mu);
        CUcontext ctx = nullptr;
        if (cudaSetDevice(dev) != cudaSuccess || !current_context(&ctx) || !ctx) return OF_ERR_CUDA;
        if (!g_slot[dev].ptr || g_slot[dev].ctx != ctx) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return OF_ERR_CUDA;
            g_slot[dev].ptr = static_cast<double*>(p);
            g_slot[dev].ctx = ctx;
        }
        scratch = g_slot[dev].ptr;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the arrival counter must start at zero (an earlier failed call may have left it set)
    if (cudaMemsetAsync(scratch + NA_COUNTER, 0, sizeof(double), st) != cudaSuccess) return OF_ERR_CUDA;
    k_residual_noalloc<<<(unsigned)nblk, NA_NW * 32, 0, st>>>(W, H, nbx, f1, f2, alpha, lambda, U, r, norms, scratch);
    if (cudaGetLastError() != cudaSuccess) return OF_ERR_CUDA;
    return OF_OK;
}
