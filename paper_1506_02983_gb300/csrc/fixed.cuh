// fixed.cuh -- the fixed-point frame of the exact constant-coefficient operator: an iterate x
// is written as X 2^-s with 64-bit integers X, s chosen per level from max |x| so that every
// |X| < 2^53 (jcg.cu, res_cc.cu).
#pragma once

#include <cuda_runtime.h>

namespace ecmg {
namespace fx {

// Per-level scale: the bit pattern of max |x| (k_absmax), read by every block.
struct FixedFrame {
    int s;          // x = X 2^-s
    double inv;     // 2^-s
    bool finite;    // false when x holds an Inf or NaN
};
__device__ __forceinline__ FixedFrame fixed_frame(unsigned long long bits)
{
    FixedFrame f;
    const int E = (int)((bits >> 52) & 0x7ff);  // biased exponent of max |x|
    f.finite = E != 0x7ff;
    f.s = (bits == 0ull || !f.finite) ? 0 : 1075 - E;  // max |x| < 2^(E-1022), so max |X| < 2^53
    f.inv = ldexp(1.0, -f.s);
    return f;
}
// X = trunc(x 2^s) from the bits of x (integer operations only; |x| <= max |x| keeps the shift
// non-positive).
__device__ __forceinline__ long long to_fixed(double x, int s)
{
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    const long long m = (b & 0xfffffffffffffll) | 0x10000000000000ll;
    const int sh = e - 1075 + s;
    long long v = 0;
    if (e != 0 && sh > -64) v = sh >= 0 ? (long long)((unsigned long long)m << sh) : (m >> -sh);
    return b < 0 ? -v : v;
}

// Exact widening of an FP32 value to FP64 by rebiasing its exponent field (integer operations;
// the conversion instruction runs on the FP64 pipe, 1/64 of the FP32 rate on GB300). Zeros
// keep their sign; subnormals, Inf and NaN take the conversion instruction.
__device__ __forceinline__ double widen(float f)
{
    const unsigned int b = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    if ((b & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sign);
    const unsigned int ex = (b >> 23) & 0xffu;
    if (ex == 0u || ex == 0xffu) return (double)f;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(ex + 896u) << 52) |
                                            ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// Bit pattern of |x| as an unsigned integer (sign bit cleared with an integer AND: fabs on a
// double would take an FP64-pipe instruction). Patterns of nonnegative doubles order like the
// values, Inf and NaN above every finite value.
__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

}  // namespace fx
}  // namespace ecmg
