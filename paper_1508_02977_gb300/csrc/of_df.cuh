// Double-float ("float-float") arithmetic for the outer residual of the
// FP32 path.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The operations are the classical error-free
// transformations: Knuth's TwoSum (exact a + b = s + e for any a, b),
// Dekker's FastTwoSum (the same when |a| >= |b|) and the FMA form of
// Dekker's TwoProduct (p = fl(a b), e = fma(a, b, -p), a b = p + e exactly).
// The sum below is the short variant (one TwoSum on the high parts, the low
// parts added in float): its absolute error is a small multiple of
// 2^-46 (|a| + |b|), which is the measure that matters for r = b - A x (the
// error relative to |b| + |A| |x|).  The FP32 pipe runs these at the full
// FP32 rate; FP64 arithmetic runs at a small fraction of it on this GPU.
//
// Every primitive uses the _rn intrinsics so that the compiler neither
// contracts a product into a later sum nor reassociates.
#pragma once

namespace ofk {

struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float v = __fsub_rn(s, a);
    return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v))};
}

__device__ __forceinline__ DF operator+(DF a, DF b) {
    const DF s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF operator-(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}

// double -> double-float: hi is x rounded to float, lo the rounded remainder
__device__ __forceinline__ DF df_from_double_fp64(double x) {
    const float h = __double2float_rn(x);
    return DF{h, __double2float_rn(x - (double)h)};
}

// Out-of-line forms of the FP64 routes below, for the rare inputs they
// serve: inlined, the compiler may execute them under a predicate for every
// input, which puts FP64 instructions on every call.
static __device__ __noinline__ DF df_from_double_slow(double x) { return df_from_double_fp64(x); }
static __device__ __noinline__ float f32_from_double_slow(double x) { return __double2float_rn(x); }

// The same from the bits of x with integer and FP32 instructions (the
// double <-> float conversions and the subtraction above run on the FP64
// pipe, a small fraction of the FP32 rate on this GPU).  x = (-1)^s 1.m 2^e
// with a 53-bit significand M: hi keeps the top 24 bits rounded to nearest
// even, and the remainder M - (top 24 bits, rounded) 2^29 (a 30-bit signed
// integer times 2^(e - 52)) is rounded to float by the int -> float
// conversion and scaled by an exact power of two.  Zeros are exact; values
// whose remainder would leave the normal float range (|x| < 2^-63 or
// |x| >= 2^127), infinities and NaNs take the FP64 route.
__device__ __forceinline__ DF df_from_double(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned s = (unsigned)(b >> 63);
    const int E = (int)((b >> 52) & 0x7ffULL);
    if ((b << 1) == 0ULL) return DF{s ? -0.0f : 0.0f, 0.0f};
    if (E < 960 || E > 1150) return df_from_double_slow(x);
    const unsigned long long m = (b & 0xfffffffffffffULL) | (1ULL << 52);
    const unsigned top = (unsigned)(m >> 29);              // 24 bits, bit 23 the implicit one
    const unsigned rest = (unsigned)(m & 0x1fffffffULL);   // 29 bits
    const bool up = rest > (1u << 28) || (rest == (1u << 28) && (top & 1u));
    const unsigned hb = (((unsigned)(E - 1023 + 127) << 23) + (top & 0x7fffffu) + (up ? 1u : 0u)) | (s << 31);
    const int ri = up ? (int)rest - (1 << 29) : (int)rest;
    const float scale = __uint_as_float((unsigned)(E - 1075 + 127) << 23);  // 2^(e - 52)
    const float lo = __fmul_rn(__int2float_rn(ri), scale);
    return DF{__uint_as_float(hb), s ? -lo : lo};
}

// double -> float, rounded to nearest even, from the bits of x with integer
// instructions (the hardware conversion runs on the FP64 pipe).  A normal
// float result (2^-126 <= |x| < 2^128 before rounding) keeps the top 24
// bits of the significand, rounded by the 29 bits below them; a carry out of
// the significand moves into the exponent field, which is the correctly
// rounded result (up to infinity above the largest float).  Zeros are
// exact; subnormal results, infinities and NaNs take the hardware route.
__device__ __forceinline__ float f32_from_double(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned s = (unsigned)(b >> 63);
    const int E = (int)((b >> 52) & 0x7ffULL);
    if ((b << 1) == 0ULL) return s ? -0.0f : 0.0f;
    if (E < 1023 - 126 || E > 1023 + 127) return f32_from_double_slow(x);
    const unsigned long long m = b & 0xfffffffffffffULL;   // 52 fraction bits
    const unsigned top = (unsigned)(m >> 29);               // 23 fraction bits kept
    const unsigned rest = (unsigned)(m & 0x1fffffffULL);    // 29 bits dropped
    const bool up = rest > (1u << 28) || (rest == (1u << 28) && (top & 1u));
    return __uint_as_float(((((unsigned)(E - 1023 + 127) << 23) | top) + (up ? 1u : 0u)) | (s << 31));
}

__device__ __forceinline__ DF shfl_down(DF v, int d) {
    return DF{__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d)};
}

// Conversions between the storage types (float, double) and an arithmetic
// type T (float, double or DF).
template <typename T>
struct Cvt {
    template <typename S>
    __device__ __forceinline__ static T from(S x) { return (T)x; }
    __device__ __forceinline__ static T from(DF x) { return (T)x.hi + (T)x.lo; }
};
template <>
struct Cvt<DF> {
    __device__ __forceinline__ static DF from(float x) { return DF{x, 0.f}; }
    __device__ __forceinline__ static DF from(double x) { return df_from_double(x); }
    __device__ __forceinline__ static DF from(DF x) { return x; }
};

// ---- Fixed-order reductions of FP64 partial sums in double-float ----------
// (the FP64 pipe of this GPU runs at a small fraction of the FP32 rate; the
// partials are read with df_from_double, integer and FP32 instructions only)

__device__ __forceinline__ DF df_warp_sum(DF v) {
    for (int o = 16; o > 0; o >>= 1)
        v = v + DF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    return v;
}

__device__ __forceinline__ double df_to_double(DF v) { return (double)v.hi + (double)v.lo; }
static __device__ __noinline__ double df_to_double_slow(DF v) { return df_to_double(v); }

// hi + lo as a double from the bits of the two floats, with integer
// instructions.  hi = (-1)^s m_h 2^(e_h - 150) with a 24-bit m_h; in units of
// 2^(e_h - 179) it is m_h 2^29, a 53-bit significand, and lo (|lo| <= ulp(hi)
// / 2, so e_l <= e_h - 24) is m_l 2^(e_l - e_h + 29), added with its sign
// (the bits of lo below the unit are dropped: an error below 2^-52 |hi|, far
// under the 2^-46 of the double-float itself).  The sum lies in [2^52 - 2^28,
// 2^53); below 2^52 it is shifted up one place.  A zero hi gives zero; a
// subnormal, infinite or NaN hi, or a lo that is not a normal float or zero,
// takes the FP64 route.
__device__ __forceinline__ double df_to_double_bits(DF v) {
    const unsigned uh = __float_as_uint(v.hi), ul = __float_as_uint(v.lo);
    const int eh = (int)((uh >> 23) & 0xffu), el = (int)((ul >> 23) & 0xffu);
    const bool lo_zero = (ul << 1) == 0u;
    if ((uh << 1) == 0u) return 0.0;
    if (eh == 0 || eh == 0xff || (!lo_zero && (el == 0 || el == 0xff))) return df_to_double_slow(v);
    long long M = (long long)((uh & 0x7fffffu) | 0x800000u) << 29;
    if (!lo_zero) {
        const long long ml = (long long)((ul & 0x7fffffu) | 0x800000u);
        const int sh = el - eh + 29;
        const long long add = sh >= 0 ? (ml << sh) : (sh > -25 ? (ml >> (-sh)) : 0LL);
        M = ((uh ^ ul) >> 31) ? M - add : M + add;
    }
    int e = eh - 127 + 1023;
    if (M < (1LL << 52)) {
        M <<= 1;
        e -= 1;
    }
    const unsigned long long bits = ((unsigned long long)(uh >> 31) << 63) | ((unsigned long long)e << 52) |
                                    ((unsigned long long)M & 0xfffffffffffffULL);
    return __longlong_as_double((long long)bits);
}

// Deterministic block sum of one double-float per thread (fixed tree order);
// the result is valid in thread 0.  sh: NT / 32 DF of shared memory.
template <int NT> __device__ __forceinline__ DF df_block_sum(DF v, DF* sh) {
    v = df_warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    DF s{0.f, 0.f};
    if (threadIdx.x < 32) {
        s = (l < NT / 32) ? sh[l] : DF{0.f, 0.f};
        s = df_warp_sum(s);
    }
    return s;
}

// This thread's share of sum_i p[i * stride], i = t, t + nt, ... < n, in K
// accumulators (element k of the share into accumulator k mod K, so that K
// loads are in flight), combined in a fixed order.
template <int K>
__device__ __forceinline__ DF df_strided_sum(const double* p, int n, int stride, int t, int nt) {
    DF a[K];
#pragma unroll
    for (int u = 0; u < K; ++u) a[u] = DF{0.f, 0.f};
    int i = t;
    for (; i + (K - 1) * nt < n; i += K * nt) {
        double v[K];
#pragma unroll
        for (int u = 0; u < K; ++u) v[u] = __ldcg(p + (long long)(i + u * nt) * stride);
#pragma unroll
        for (int u = 0; u < K; ++u) a[u] = a[u] + df_from_double(v[u]);
    }
#pragma unroll
    for (int u = 0; u < K - 1; ++u)
        if (i + u * nt < n) a[u] = a[u] + df_from_double(__ldcg(p + (long long)(i + u * nt) * stride));
#pragma unroll
    for (int w = 1; w < K; w <<= 1)
#pragma unroll
        for (int u = 0; u + w < K; u += 2 * w) a[u] = a[u] + a[u + w];
    return a[0];
}

// The sums of the two interleaved streams p[2 i] and p[2 i + 1], i < n (p
// 16-byte aligned), in a fixed order by one block: per thread as in
// df_strided_sum (K accumulators per stream, one 16-byte load per i), then a
// fixed tree over each warp and over the warps.  Every thread of the block
// calls it; the results are those of thread 0.  sh: 64 DF of shared memory,
// free on entry.
template <int K>
__device__ __forceinline__ void df_ordered_sum2(const double* p, int n, double& s0, double& s1, DF* sh) {
    const int nt = blockDim.x, t = threadIdx.x;
    const double2* q = reinterpret_cast<const double2*>(p);
    DF a[K], b[K];
#pragma unroll
    for (int u = 0; u < K; ++u) a[u] = b[u] = DF{0.f, 0.f};
    int i = t;
    for (; i + (K - 1) * nt < n; i += K * nt) {
        double2 v[K];
#pragma unroll
        for (int u = 0; u < K; ++u) v[u] = __ldcg(q + i + u * nt);
#pragma unroll
        for (int u = 0; u < K; ++u) {
            a[u] = a[u] + df_from_double(v[u].x);
            b[u] = b[u] + df_from_double(v[u].y);
        }
    }
#pragma unroll
    for (int u = 0; u < K - 1; ++u)
        if (i + u * nt < n) {
            const double2 v = __ldcg(q + i + u * nt);
            a[u] = a[u] + df_from_double(v.x);
            b[u] = b[u] + df_from_double(v.y);
        }
#pragma unroll
    for (int w = 1; w < K; w <<= 1)
#pragma unroll
        for (int u = 0; u + w < K; u += 2 * w) {
            a[u] = a[u] + a[u + w];
            b[u] = b[u] + b[u + w];
        }
    DF x = a[0], y = b[0];
    x = df_warp_sum(x);
    y = df_warp_sum(y);
    const int w = t >> 5, l = t & 31;
    __syncthreads();
    if (l == 0) {
        sh[w] = x;
        sh[32 + w] = y;
    }
    __syncthreads();
    if (t < 32) {
        const int nw = (nt + 31) >> 5;
        x = l < nw ? sh[l] : DF{0.f, 0.f};
        y = l < nw ? sh[32 + l] : DF{0.f, 0.f};
        x = df_warp_sum(x);
        y = df_warp_sum(y);
        if (t == 0) {
            s0 = df_to_double(x);
            s1 = df_to_double(y);
        }
    }
}

// A constant in type T, evaluated by the compiler (the callers bind it to a
// constexpr variable, so that no FP64 instruction forms it at run time).
template <typename T> __host__ __device__ constexpr T kconst(double x) { return (T)x; }
template <> __host__ __device__ constexpr DF kconst<DF>(double x) {
    return DF{(float)x, (float)(x - (double)(float)x)};
}

}  // namespace ofk
