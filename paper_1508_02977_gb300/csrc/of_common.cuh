// Shared device-side definitions of the optical-flow solver (sm_103a).
//
// Discretisation (Section 2.2, Fig. sch-mesh): one node per pixel centre,
// square (x,y) cut along (x,y)->(x+1,y+1) into
//   t=0: a=(x,y) b=(x+1,y) c=(x+1,y+1)     t=1: a=(x,y) d=(x,y+1) c=(x+1,y+1)
// with |K| = 1/2.  Per element the data of Eq. OF2 are
//   g = (d/dx f2_h, d/dy f2_h, -mean f1),   ft = mean (f2 - f1)
// and the element matrix of the weak form (Eq. discret-form) is
//   |K|/12 (1+delta_ij) g g^T  +  |K| Lambda grad phi_i . grad phi_j,
// Lambda = (alpha_K, alpha_K, lambda), load -|K|/3 ft g.  On these right
// triangles the stiffness couples only the two legs of each triangle, each
// with weight |K| = 1/2, so the node stencil is 7-point.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ofk {

// Workspace layouts (device):
//   frame  [H][pitch]          Real
//   alpha  [H][pitch][2]       Real   (square (x,y) of rows 0..H-2, cols 0..W-2)
//   vector [3][H][pitch]       Real   (plane stride H*pitch)
struct PairDesc {
    int W, H, pitch;
    int tiles_x, tiles_y;   // Schwarz tiles of this pair
    int tile0;              // first Schwarz work item of this pair
    int blk0, nblk;         // first apply block of this pair, number of apply blocks
    long long frame_off;    // element offset of this pair's frames in the frame arrays
    long long vec_off;      // element offset of this pair's planes in the vector arrays
    long long pair_off;     // element offset of this pair's paired element records (FP16 sweeps):
                            // [H + ov + 1][pitch], row k holding the records of image row k - ov - 1
};

// Per-pair scalars of the Krylov loop (device memory, FP64).
struct PairScalars {
    double rz;        // r.z of the current iterate
    double pq;        // p.q
    double a;         // step a = rz / pq of the current iteration
    double a_prev;    // step of the previous iteration (deferred x update)
    double beta;      // rz_new / rz_old
    double rr;        // ||r||^2 of the inner (recursive) residual
    double tol2;      // inner stop: rr <= tol2
    double bnorm2;    // ||b||^2 (FP64)
    double res2;      // ||b - A x||^2 of the last FP64 residual evaluation
    int it;           // inner iterations done in this pass
    int it_total;     // inner iterations in total
    int done;         // inner loop finished (converged, capped or broken down)
    int status;       // 0 ok, 5 not converged, 6 breakdown
    int max_it;       // inner iteration cap of this pass
    int pad[3];       // pad[0]: outer convergence; pad[1]: a p.q partial was not finite or too large
    long long pq_fix; // FP32 path, one pair: p.q as a fixed-point integer sum (pq_fix_shift)
};

// p.q of the FP32 PCG apply as a sum of 64-bit integers (one pair, FP16
// sweeps): each apply block adds its FP32 partial times 2^k, rounded to an
// integer, k = 40 minus the binary exponent of r.z (clamped to the range of a
// float power of two).  Integer addition is exact and independent of the
// order, so the sum is deterministic without a reduction tree or an arrival
// count; the preconditioner kernel that follows reads it after the launch
// boundary.  The rounding error of the sum is below (blocks / 2) 2^-40 |r.z|;
// it overflows only when the partials' magnitudes add up to 2^22 |r.z| (p.q =
// r.z / a with a of order one for a preconditioned system).
__device__ __forceinline__ int pq_fix_shift(double rz) {
    const int e = (int)(((unsigned long long)__double_as_longlong(rz) >> 52) & 0x7ffULL) - 1023;
    const int k = 40 - e;
    return k < -126 ? -126 : (k > 127 ? 127 : k);
}

#define OF_STIFF_HALF 0.5   // |K| * |grad phi|^2 weight of a triangle leg

// Device index checks, compiled in with -DOF_BOUNDS_CHECK (a separate build of
// the library that the tests run): an index outside [0, n) sets bit 2 of the
// device error word and the access it guards is skipped (no trap); the entry
// point then returns OF_ERR_CUDA.  Without the flag a check is the constant
// true and costs nothing.
constexpr int OF_ERR_BIT_BOUNDS = 4;
#ifdef OF_BOUNDS_CHECK
__device__ __forceinline__ bool of_in_range(int* err, long long i, long long n) {
    if (i >= 0 && i < n) return true;
    if (err) atomicOr(err, OF_ERR_BIT_BOUNDS);
    return false;
}
#define OF_CHECK(err, i, n) ofk::of_in_range((err), (long long)(i), (long long)(n))
#else
#define OF_CHECK(err, i, n) true
#endif

template <typename T> __device__ __forceinline__ T ld_or0(const T* p, bool ok) { return ok ? *p : T(0); }

__device__ __forceinline__ float shfl_down(float v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_down(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v) {
    for (int o = 16; o > 0; o >>= 1) { T w = __shfl_xor_sync(0xffffffffu, v, o); v = w > v ? w : v; }
    return v;
}

// Deterministic block sum of one double per thread (fixed tree order).
template <int NT> __device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (l < NT / 32) ? sh[l] : 0.0;
        s = warp_sum(s);
    }
    return s;  // valid in thread 0
}

// "Last block of the pair" protocol: every block writes its partial, fences,
// and bumps the pair counter; the block that sees count == n-1 reduces all
// partials of the pair in index order (deterministic) and resets the
// counter for the next launch.
// The arrival is one acquire-release atomic at GPU scope by thread 0: its
// release covers the block's writes (ordered before it by the barrier), its
// acquire the other blocks' writes for every thread of the last block
// (ordered after it by the second barrier).
__device__ __forceinline__ bool arrive_last(unsigned* counter, unsigned n, int* sh_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(prev) : "l"(counter), "r"(1u) : "memory");
        *sh_flag = (prev == n - 1) ? 1 : 0;
    }
    __syncthreads();
    return *sh_flag != 0;
}

// Sum of n doubles (stride `stride`) in fixed order by one block.
// This thread's share of p[i * stride], i = t, t + nt, ... < n: eight
// accumulators (element k of the share goes to accumulator k mod 8) so that
// eight loads are in flight, combined in a fixed order.
__device__ __forceinline__ double strided_sum8(const double* p, int n, int stride, int t, int nt) {
    double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int i = t;
    for (; i + 7 * nt < n; i += 8 * nt) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] += __ldcg(p + (long long)(i + u * nt) * stride);
    }
#pragma unroll
    for (int u = 0; u < 7; ++u)
        if (i + u * nt < n) a[u] += __ldcg(p + (long long)(i + u * nt) * stride);
    return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

template <int NT> __device__ double ordered_sum(const double* p, int n, int stride, double* sh) {
    return block_sum<NT>(strided_sum8(p, n, stride, threadIdx.x, NT), sh);
}

}  // namespace ofk
