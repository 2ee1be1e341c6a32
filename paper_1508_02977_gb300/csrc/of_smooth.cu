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

template <typename D, bool TRANS>
__global__ void k_smooth_axis(const D* __restrict__ in, D* __restrict__ out, int W, int H, long long pitch, int axis,
                              const SmoothTaps T) {
    __shared__ D sw[2 * OF_SMOOTH_RMAX + 1], scw[2 * OF_SMOOTH_RMAX + 2];
    const int r = T.r;
    for (int j = threadIdx.x; j <= 2 * r + 1; j += blockDim.x) {
        if (j <= 2 * r) sw[j] = (D)T.w[j];
        scw[j] = (D)T.cw[j];
    }
    __syncthreads();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    const int n = axis == 0 ? W : H;
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
        const int pos = axis == 0 ? x : y;
        const int lo = max(-r, -pos), hi = min(r, n - 1 - pos);
        const long long step = axis == 0 ? 1 : pitch;
        const D* src = in + (long long)y * pitch + x;
        D acc = D(0);
        for (int k = lo; k <= hi; ++k) {
            D v = src[k * step];
            if (TRANS) {
                const int q = pos + k;  // normaliser of the output position that tap feeds
                v = v / tap_sum<D>(scw, r, max(-r, -q), min(r, n - 1 - q));
            }
            acc += sw[k + r] * v;
        }
        if (!TRANS) acc = acc / tap_sum<D>(scw, r, lo, hi);
        out[(long long)y * pitch + x] = acc;
    }
}

template <typename D>
static cudaError_t smooth_t(D* f, D* scratch, int W, int H, long long pitch, const SmoothTaps& T, bool transpose,
                            cudaStream_t st) {
    const dim3 block(128), grid((W + 127) / 128, H < 65535 ? H : 65535);
    if (!transpose) {  // S = S_y S_x
        k_smooth_axis<D, false><<<grid, block, 0, st>>>(f, scratch, W, H, pitch, 0, T);
        k_smooth_axis<D, false><<<grid, block, 0, st>>>(scratch, f, W, H, pitch, 1, T);
    } else {           // S^T = S_x^T S_y^T
        k_smooth_axis<D, true><<<grid, block, 0, st>>>(f, scratch, W, H, pitch, 1, T);
        k_smooth_axis<D, true><<<grid, block, 0, st>>>(scratch, f, W, H, pitch, 0, T);
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
