// Device helpers shared by the kernels of the mf library: the status word
// and the fixed-point to FP64 conversion of the mixed elasticity path.
#pragma once

// device status codes are written with atomicCAS(word, 0, code): first error wins
__device__ __forceinline__ void mf_dev_fail(int *word, int code) { atomicCAS(word, 0, code); }

// x * 2^-S for a fixed-point integer x, rounded to nearest even with integer
// operations only (no FP64 instruction: FP64 runs at 1/58 of FP32 here).
__device__ __forceinline__ double mf_fixed_to_double(long long v, int S)
{
    if (v == 0) return 0.0;
    const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
    unsigned long long u = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
    const int lz = __clzll((long long)u);
    u <<= lz;  // leading one at bit 63
    unsigned long long m = u >> 11;  // 53 significant bits
    const unsigned long long rest = u & 0x7ffull;
    m += (rest > 0x400ull || (rest == 0x400ull && (m & 1ull))) ? 1ull : 0ull;
    const long long ex = 1023 + (63 - lz) - S;
    if (ex <= 0) return __longlong_as_double((long long)sign);  // below the normal range
    const unsigned long long bits = ((unsigned long long)ex << 52) + (m - (1ull << 52));
    return __longlong_as_double((long long)(bits | sign));
}
