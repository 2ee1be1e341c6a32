// Gaussian pre-smoothing of the frames, f = K_sigma * I (Section 1), and its
// transpose for the frame gradients of the adjoint; the K_rho element
// tensors A_rho = K_rho * (g g^T), F = K_rho * (-ft g) of Section 1.
//
// Discrete K_sigma: the sampled Gaussian w_k = exp(-k^2 / (2 sigma^2)),
// |k| <= r = ceil(3 sigma), applied along x and then along y.  Each pass is
// normalised over the taps that fall inside the image,
//   (S_x I)(x) = sum_{k : 0 <= x+k < W} w_k I(x+k) / N(x),  N(x) = sum of those w_k,
// so constants are preserved and nothing outside the image is invented.
// S = S_y S_x; its transpose S^T = S_x^T S_y^T with
//   (S_x^T g)(x) = sum_{k : 0 <= x+k < W} w_k g(x+k) / N(x+k).
#include <cuda_runtime.h>

#include "of_launch.h"

namespace ofl {

// The taps in the storage type, staged in shared memory once per block (an
// FP64 -> FP32 conversion per tap and output would run on the FP64 pipe).
// tap_sum: the weights of offsets lo..hi from the prefix table
// cw[i] = w_0 + ... + w_{i-1} (w_j the weight of offset j - r).
template <typename D>
__device__ __forceinline__ D tap_sum(const D* cw, int r, int lo, int hi) { return cw[hi + r + 1] - cw[lo + r]; }

// The pass along x: a block takes 128 columns of SMOOTH_SX rows; the taps
// and their bounds depend on x only, so the rows accumulate side by side
// (independent loads in flight).
constexpr int SMOOTH_SX = 8;
template <typename D, bool TRANS>
__global__ void __launch_bounds__(128) k_smooth_x(const D* __restrict__ in, D* __restrict__ out, int W, int H,
                                                  long long pitch, const SmoothTaps T) {
    __shared__ D sw[2 * OF_SMOOTH_RMAX + 1], scw[2 * OF_SMOOTH_RMAX + 2];
    const int r = T.r;
    for (int j = threadIdx.x; j <= 2 * r + 1; j += blockDim.x) {
        if (j <= 2 * r) sw[j] = (D)T.w[j];
        scw[j] = (D)T.cw[j];
    }
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    const int y0 = blockIdx.y * SMOOTH_SX, ny = min(SMOOTH_SX, H - y0);
    const int lo = max(-r, -x), hi = min(r, W - 1 - x);
    D acc[SMOOTH_SX];
#pragma unroll
    for (int u = 0; u < SMOOTH_SX; ++u) acc[u] = D(0);
    const D* src = in + (long long)y0 * pitch + x;
    for (int k = lo; k <= hi; ++k) {
        D wk = sw[k + r];
        if (TRANS) {
            const int q = x + k;  // normaliser of the output position that tap feeds
            wk = wk / tap_sum<D>(scw, r, max(-r, -q), min(r, W - 1 - q));
        }
#pragma unroll
        for (int u = 0; u < SMOOTH_SX; ++u)
            if (u < ny) acc[u] += wk * src[(long long)u * pitch + k];
    }
    const D nrm = TRANS ? D(1) : tap_sum<D>(scw, r, lo, hi);
#pragma unroll
    for (int u = 0; u < SMOOTH_SX; ++u)
        if (u < ny) out[(long long)(y0 + u) * pitch + x] = TRANS ? acc[u] : acc[u] / nrm;
}

// The pass along y: a block stages a strip of SMOOTH_SY rows (plus r rows
// above and below) of 128 columns in shared memory with coalesced loads, then
// each thread walks its column; every input is read once per strip instead
// of once per tap.  The transposed pass divides each input by the normaliser
// of its own position while staging it.
constexpr int SMOOTH_SY = 64;
template <typename D>
__host__ __device__ constexpr size_t smooth_y_smem(int r) { return (size_t)(SMOOTH_SY + 2 * r) * 128 * sizeof(D); }

template <typename D, bool TRANS>
__global__ void __launch_bounds__(128) k_smooth_y(const D* __restrict__ in, D* __restrict__ out, int W, int H,
                                                  long long pitch, const SmoothTaps T) {
    extern __shared__ __align__(16) unsigned char ysm[];
    D* tile = reinterpret_cast<D*>(ysm);  // [(SMOOTH_SY + 2 r)][128]
    __shared__ D sw[2 * OF_SMOOTH_RMAX + 1], scw[2 * OF_SMOOTH_RMAX + 2];
    const int r = T.r, tid = threadIdx.x;
    for (int j = tid; j <= 2 * r + 1; j += blockDim.x) {
        if (j <= 2 * r) sw[j] = (D)T.w[j];
        scw[j] = (D)T.cw[j];
    }
    __syncthreads();
    const int x = blockIdx.x * 128 + tid, y0 = blockIdx.y * SMOOTH_SY;
    const int ylo = max(y0 - r, 0), yhi = min(y0 + SMOOTH_SY + r, H);
#pragma unroll 8
    for (int yy = ylo; yy < yhi; ++yy) {  // eight rows' loads in flight
        D v = D(0);
        if (x < W) {
            v = in[(long long)yy * pitch + x];
            if (TRANS) v = v / tap_sum<D>(scw, r, max(-r, -yy), min(r, H - 1 - yy));
        }
        tile[(yy - ylo) * 128 + tid] = v;
    }
    __syncthreads();
    if (x >= W) return;
    const int yend = min(y0 + SMOOTH_SY, H);
    for (int y = y0; y < yend; ++y) {
        const int lo = max(-r, -y), hi = min(r, H - 1 - y);
        D acc = D(0);
        for (int k = lo; k <= hi; ++k) acc += sw[k + r] * tile[(y + k - ylo) * 128 + tid];
        if (!TRANS) acc = acc / tap_sum<D>(scw, r, lo, hi);
        out[(long long)y * pitch + x] = acc;
    }
}

template <typename D>
static cudaError_t smooth_t(D* f, D* scratch, int W, int H, long long pitch, const SmoothTaps& T, bool transpose,
                            cudaStream_t st) {
    const dim3 block(128);
    const dim3 gy((W + 127) / 128, (H + SMOOTH_SY - 1) / SMOOTH_SY);
    const size_t sy = smooth_y_smem<D>(T.r);
    static bool attr_set = false;  // the largest strip (r = OF_SMOOTH_RMAX) needs the opt-in size
    if (!attr_set) {
        const int mx = (int)smooth_y_smem<D>(OF_SMOOTH_RMAX);
        cudaFuncSetAttribute(k_smooth_y<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_smooth_y<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        attr_set = true;
    }
    const dim3 gx((W + 127) / 128, (H + SMOOTH_SX - 1) / SMOOTH_SX);
    if (!transpose) {  // S = S_y S_x
        k_smooth_x<D, false><<<gx, block, 0, st>>>(f, scratch, W, H, pitch, T);
        k_smooth_y<D, false><<<gy, block, sy, st>>>(scratch, f, W, H, pitch, T);
    } else {           // S^T = S_x^T S_y^T
        k_smooth_y<D, true><<<gy, block, sy, st>>>(f, scratch, W, H, pitch, T);
        k_smooth_x<D, true><<<gx, block, 0, st>>>(scratch, f, W, H, pitch, T);
    }
    return cudaGetLastError();
}

// Products of the element data of square (x, y): planes t * 9 + k, k = 0..5
// the entries 00, 01, 02, 11, 12, 22 of g g^T, k = 6..8 the load -ft g, with
// g = (d/dx f2_h, d/dy f2_h, -gms mean f1) and ft = mean (f2 - f1) over the
// triangle's vertices (t = 0: (x,y), (x+1,y), (x+1,y+1); t = 1: (x,y),
// (x,y+1), (x+1,y+1)).
template <typename D>
__global__ void k_eld_products(const D* __restrict__ f1, const D* __restrict__ f2, int W, int H, long long pitch,
                               D gms, D* __restrict__ eld, long long stride) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W - 1) return;
    const D third = D(1) / D(3);
    for (int y = blockIdx.y; y < H - 1; y += gridDim.y) {
        const long long o = (long long)y * pitch + x;
        const D a1 = f1[o], b1 = f1[o + 1], c1 = f1[o + pitch + 1], d1 = f1[o + pitch];
        const D a2 = f2[o], b2 = f2[o + 1], c2 = f2[o + pitch + 1], d2 = f2[o + pitch];
        const D g[2][3] = {{b2 - a2, c2 - b2, -(a1 + b1 + c1) * third * gms},
                           {c2 - d2, d2 - a2, -(a1 + d1 + c1) * third * gms}};
        const D ft[2] = {((a2 - a1) + (b2 - b1) + (c2 - c1)) * third, ((a2 - a1) + (d2 - d1) + (c2 - c1)) * third};
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            D* e = eld + o + (long long)(9 * t) * stride;
            e[0 * stride] = g[t][0] * g[t][0];
            e[1 * stride] = g[t][0] * g[t][1];
            e[2 * stride] = g[t][0] * g[t][2];
            e[3 * stride] = g[t][1] * g[t][1];
            e[4 * stride] = g[t][1] * g[t][2];
            e[5 * stride] = g[t][2] * g[t][2];
            e[6 * stride] = -ft[t] * g[t][0];
            e[7 * stride] = -ft[t] * g[t][1];
            e[8 * stride] = -ft[t] * g[t][2];
        }
    }
}

cudaError_t launch_element_data(const void* f1, const void* f2, int type, int W, int H, long long pitch, double gms,
                                void* eld, long long stride, void* scratch, const SmoothTaps& T, cudaStream_t st) {
    if (W < 2 || H < 2) return cudaSuccess;
    const dim3 block(128), grid((W - 1 + 127) / 128, H - 1 < 65535 ? H - 1 : 65535);
    if (type == T_F64)
        k_eld_products<double><<<grid, block, 0, st>>>((const double*)f1, (const double*)f2, W, H, pitch, gms,
                                                       (double*)eld, stride);
    else
        k_eld_products<float><<<grid, block, 0, st>>>((const float*)f1, (const float*)f2, W, H, pitch, (float)gms,
                                                      (float*)eld, stride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || T.r <= 0) return e;
    // K_rho over the (W-1) x (H-1) lattice of each plane
    const size_t es = type == T_F64 ? 8 : 4;
    for (int q = 0; q < 18; ++q) {
        e = launch_smooth((char*)eld + (size_t)q * stride * es, scratch, type, W - 1, H - 1, pitch, T, false, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_smooth(void* f, void* scratch, int type, int W, int H, long long pitch, const SmoothTaps& T,
                          bool transpose, cudaStream_t st) {
    if (W <= 0 || H <= 0) return cudaSuccess;
    if (type == T_F64) return smooth_t<double>((double*)f, (double*)scratch, W, H, pitch, T, transpose, st);
    return smooth_t<float>((float*)f, (float*)scratch, W, H, pitch, T, transpose, st);
}

}  // namespace ofl
