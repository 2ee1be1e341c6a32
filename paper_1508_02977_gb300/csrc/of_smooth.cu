// Gaussian pre-smoothing of the frames, f = K_sigma * I (Section 1), and its
// transpose for the frame gradients of the adjoint.
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

// sum of the weights of offsets lo..hi (prefix table cw[i] = w_0 + ... + w_{i-1},
// w_j the weight of offset j - r)
__device__ __forceinline__ double tap_sum(const SmoothTaps& T, int lo, int hi) { return T.cw[hi + T.r + 1] - T.cw[lo + T.r]; }

template <typename D, bool TRANS>
__global__ void k_smooth_axis(const D* __restrict__ in, D* __restrict__ out, int W, int H, long long pitch, int axis,
                              const SmoothTaps T) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    const int n = axis == 0 ? W : H;
    for (int y = blockIdx.y; y < H; y += gridDim.y) {
        const int pos = axis == 0 ? x : y;
        const int lo = max(-T.r, -pos), hi = min(T.r, n - 1 - pos);
        const long long step = axis == 0 ? 1 : pitch;
        const D* src = in + (long long)y * pitch + x;
        D acc = D(0);
        for (int k = lo; k <= hi; ++k) {
            D v = src[k * step];
            if (TRANS) {
                const int q = pos + k;  // normaliser of the output position that tap feeds
                v = v / (D)tap_sum(T, max(-T.r, -q), min(T.r, n - 1 - q));
            }
            acc += (D)T.w[k + T.r] * v;
        }
        if (!TRANS) acc = acc / (D)tap_sum(T, lo, hi);
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

cudaError_t launch_smooth(void* f, void* scratch, int type, int W, int H, long long pitch, const SmoothTaps& T,
                          bool transpose, cudaStream_t st) {
    if (W <= 0 || H <= 0) return cudaSuccess;
    if (type == T_F64) return smooth_t<double>((double*)f, (double*)scratch, W, H, pitch, T, transpose, st);
    return smooth_t<float>((float*)f, (float*)scratch, W, H, pitch, T, transpose, st);
}

}  // namespace ofl
