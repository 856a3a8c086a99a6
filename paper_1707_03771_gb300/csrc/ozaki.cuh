// Ozaki error-free splitting shared by the split-precision kernels: a value already scaled by its
// row's (or column's) power of two, |x| < 1, is written as sum_s m_s 2^{-7(s+1)} with integers
// m_1 in [-128, 128] and m_{s>1} in [-64, 64], each exact in BF16.
#pragma once
#include <cuda_bf16.h>

namespace dfhf {

template <int S>
__device__ __forceinline__ void split_fp64(double x, __nv_bfloat16* out, long long stride) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const double t = x * 128.0;
        const double m = rint(t);
        x = t - m;
        out[s * stride] = __float2bfloat16_rn((float)m);
    }
}

}  // namespace dfhf
