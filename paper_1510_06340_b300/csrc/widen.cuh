// widen.cuh -- FP32 -> FP64 for the FP64 sums, by the IEEE-754 bit layouts.
// On B300 the conversion instruction issues at the FP64 rate; the FP64 sums
// of an FP32 state spend as much time converting as adding. A normal float
// (biased exponent 1..254) becomes the double with the exponent rebiased from
// 127 to 1023 and the 23-bit fraction moved up by 29 bits, which is the exact
// value; zero keeps its sign. Subnormal, infinite and NaN inputs take the
// conversion instruction, so every input gives what double(x) gives.
#pragma once

__device__ __forceinline__ double widen(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned ex = (b >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    if (ex == 0u) {
        if ((b & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sign);
        return double(x);
    }
    if (ex == 0xffu) return double(x);
    const unsigned long long d = sign | ((unsigned long long)(ex + 896u) << 52) |
                                 ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)d);
}
__device__ __forceinline__ double widen(double x) { return x; }
