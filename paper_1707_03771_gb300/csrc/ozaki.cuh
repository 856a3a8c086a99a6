// Ozaki error-free splitting shared by the split-precision kernels: a value v of a row (or column)
// whose power of two is e (|v 2^-e| < 1) is written as sum_s d_s 2^{-7s} 2^e + r, |r| <= 2^{-7S-1} 2^e,
// with integer digits d_1 in [-128, 128] and d_{s>1} in [-64, 63], each exact in BF16.
#pragma once
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

namespace dfhf {

// Longest exact chunk of a product of S-slice operands, in contraction terms (a multiple of 64). The pairs
// (s, t) with s + t = L + 2 meet in level L; per term the top level S - 1 is the largest, at most
// 2 * 128 * 64 (d_1 with d_S, twice) + (S - 2) * 64 * 64 (the inner pairs) = 2^14 + (S - 2) 2^12. A chunk
// of K terms keeps every level sum an integer of magnitude <= K * that <= 2^24, exact in FP32 whatever
// the order of the tensor-core additions: 1024, 768, 640, 576 and 448 terms for S = 2, 3, 4, 5 and 7.
template <int S>
constexpr int exact_chunk() {
    return ((1 << 24) / ((1 << 14) + (S > 2 ? S - 2 : 0) * (1 << 12))) / 64 * 64;
}
static_assert(exact_chunk<3>() == 768 && exact_chunk<5>() == 576 && exact_chunk<7>() == 448, "exact chunks");

// 2^e as a double, -1022 <= e <= 1023
__device__ __forceinline__ double pow2d(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// v 2^e for any e the slices produce (two exact power-of-two factors keep each in the normal range)
__device__ __forceinline__ double scale_pow2(double v, int e) {
    const int a = e / 2;
    return (v * pow2d(a)) * pow2d(e - a);
}

// rint(v 2^k), ties to even, from the bits of v: for a normal v = m 2^{be-1075} (m the 53-bit significand)
// the scaled value is m 2^{-d} with d = 1075 - be - k, rounded by an integer shift. Exact, as the scaling by
// a power of two is; no FP64 instruction on this path (the FP64 pipe, not HBM, bounded the slicing kernels
// when the scaling and the conversion ran there). Zero gives 0; a subnormal v, or a scaled value of 2^52 or
// more, takes the FP64 route (rint of the exactly scaled value), which the slices never need.
__host__ __device__ __forceinline__ long long rint_pow2(double v, int k) {
    unsigned long long b;
    memcpy(&b, &v, sizeof b);
    if ((b << 1) == 0) return 0;
    const int be = (int)((b >> 52) & 0x7ff);
    const int d = 1075 - be - k;
    if (be == 0 || d <= 0) {
        const int a = k / 2;
        return (long long)rint(ldexp(ldexp(v, a), k - a));
    }
    if (d >= 54) return 0;                            // |v 2^k| < 2^53 2^-54 = 1/2
    const long long m = (long long)((b & 0xfffffffffffffULL) | 0x10000000000000ULL);
    long long q = m >> d;
    const long long rem = m & ((1LL << d) - 1), half = 1LL << (d - 1);
    q += (rem > half || (rem == half && (q & 1))) ? 1 : 0;
    return (b >> 63) ? -q : q;
}

// The digits come from one integer: T = rint(v 2^{7S-e}) (|T| <= 2^{7S}) peeled into balanced base-128
// digits from the least significant end (d_S..d_2 in [-64, 63], d_1 the remaining quotient). Integer
// arithmetic throughout.
template <int S>
__device__ __forceinline__ void split_pow2(double v, int e, __nv_bfloat16* out, long long stride) {
    long long T = rint_pow2(v, 7 * S - e);
#pragma unroll
    for (int s = S - 1; s >= 1; --s) {
        const int d = (int)((T + 64) & 127) - 64;
        out[s * stride] = __int2bfloat16_rn(d);
        T = (T - d) >> 7;
    }
    out[0] = __int2bfloat16_rn((int)T);
}

}  // namespace dfhf
