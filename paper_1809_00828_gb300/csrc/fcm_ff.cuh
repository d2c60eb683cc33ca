// Double-float arithmetic on the FP32 pipe and FP64 <-> FP32 conversions by integer operations
// (internal to libfcm).  GB300's FP64 pipe, which also converts between FP64 and FP32, does 2
// operations per clock per SM; these helpers let the kernels keep FP64-level accuracy without it.
// A double-float value is a float pair (hi, lo) whose exact sum is the value.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace fcm {

// ---- FP64 -> FP32 splits by integer operations
//
// GB300's FP64 pipe, which also converts between FP64 and FP32, does 2 operations per clock per SM, so
// the kernels never convert a gathered FP64 value with it.  split_bits<MB> reads the value's bits:
// hi = x with its significand cut to MB fraction bits (exact in a format with MB fraction bits), lo =
// x - hi (a 42 to 52 - MB bit integer times a power of two) rounded to MB + 1 significant bits, half
// up in magnitude.  MB = 23: a float pair with |x - hi - lo| <= 2^-48 |x|; MB = 10: two TF32 values
// with |x - hi - lo| <= 2^-22 |x|.  |x| below 2^-126 gives +-0; beyond the FP32 range +-inf (NaN
// stays NaN), as a conversion would; a lo below 2^-126 is dropped.
template <int MB>
__device__ __forceinline__ void split_bits(double x, float &hi, float &lo)
{
    constexpr int CUT = 52 - MB;  // fraction bits of x below hi
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
    const int E = (int)(u >> 52) & 0x7FF;
    const unsigned long long M = u & 0xFFFFFFFFFFFFFull;
    const int ef = E - 896;  // FP32 exponent field of x: E - 1023 + 127
    lo = 0.f;
    if (ef <= 0) {
        hi = __uint_as_float(sign);
        return;
    }
    if (ef >= 255) {
        hi = __uint_as_float(sign | (E == 0x7FF && M ? 0x7FC00000u : 0x7F800000u));
        return;
    }
    hi = __uint_as_float(sign | ((unsigned)ef << 23) | ((unsigned)(M >> CUT) << (23 - MB)));
    const unsigned long long R = M & ((1ull << CUT) - 1);  // x - hi = R 2^(E - 1075)
    if (R == 0) return;
    const int t = 63 - __clzll((long long)R);               // leading one of R
    int e = ef - 52 + t;                                    // FP32 exponent field of lo
    unsigned q;                                             // MB + 1 significant bits
    if (t > MB) {
        q = (unsigned)(((R >> (t - MB - 1)) + 1) >> 1);
        if (q == (2u << MB)) {
            q = 1u << MB;
            ++e;
        }
    } else {
        q = (unsigned)(R << (MB - t));
    }
    if (e > 0) lo = __uint_as_float(sign | ((unsigned)e << 23) | ((q & ((1u << MB) - 1)) << (23 - MB)));
}

// x as a float pair, x = hi + lo to 2^-48 relative
__device__ __forceinline__ float2 split_ff(double x)
{
    float h, l;
    split_bits<23>(x, h, l);
    return make_float2(h, l);
}

// x rounded to FP32 (the pair's sum: within half an ulp but for ties)
__device__ __forceinline__ float to_f32(double x)
{
    float h, l;
    split_bits<23>(x, h, l);
    return __fadd_rn(h, l);
}

// a gathered residual value in the factor's type
template <typename T> __device__ __forceinline__ T gathered(double x);
template <> __device__ __forceinline__ float gathered<float>(double x) { return to_f32(x); }
template <> __device__ __forceinline__ double gathered<double>(double x) { return x; }

// FP32 -> FP64 from the bits (exact; FP32 subnormals become zero)
__device__ __forceinline__ double f2d(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    const unsigned long long frac = (unsigned long long)(b & 0x7FFFFFu) << 29;
    if (e == 0) return __longlong_as_double((long long)sign);
    if (e == 0xFF) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull | frac));
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896) << 52) | frac));
}

// ---- double-float arithmetic (FP32 pipe)

// S + C += (fh + fl)(xh + xl): the product fh xh exactly as p + e (FMA), the cross terms in FP32,
// fl xl (2^-48 relative) dropped; S accumulates by TwoSum, its rounding errors go to C.  The
// intrinsics keep the compiler from contracting or reassociating these steps.
__device__ __forceinline__ void ff_fma(float fh, float fl, float xh, float xl, float &S, float &C)
{
    const float p = __fmul_rn(fh, xh);
    const float e = __fmaf_rn(fh, xh, -p);
    C = __fmaf_rn(fh, xl, C);
    C = __fmaf_rn(fl, xh, C);
    C = __fadd_rn(C, e);
    const float s = __fadd_rn(S, p);
    const float bb = __fsub_rn(s, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    S = s;
    C = __fadd_rn(C, err);
}

// (S, C) += (S2, C2) with S by TwoSum (symmetric in the two operands)
__device__ __forceinline__ void ff_add(float &S, float &C, float S2, float C2)
{
    const float s = __fadd_rn(S, S2);
    const float bb = __fsub_rn(s, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bb)), __fsub_rn(S2, bb));
    S = s;
    C = __fadd_rn(__fadd_rn(C, C2), err);
}


// (hi, lo) with hi = fl(s + c), lo the rounding error (Fast2Sum; |s| >= |c| or s = 0)
__device__ __forceinline__ float2 ff_norm(float s, float c)
{
    const float h = __fadd_rn(s, c);
    return make_float2(h, __fsub_rn(c, __fsub_rn(h, s)));
}

// a * b for double-floats (Dekker's product with FMA; the lo * lo term dropped)
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    return ff_norm(p, e);
}

// a + b for double-floats (TwoSum of the high parts)
__device__ __forceinline__ float2 ff_addv(float2 a, float2 b)
{
    float s = a.x, c = a.y;
    ff_add(s, c, b.x, b.y);
    return ff_norm(s, c);
}

// the double closest to hi + lo (two exact widenings, one FP64 add)
__device__ __forceinline__ double ff_to_double(float2 v) { return f2d(v.x) + f2d(v.y); }

}  // namespace fcm
