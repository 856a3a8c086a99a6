// Metric whitening B = L^-1 (Q|mu nu) (paper eq. 1, third form, with M' = L^-1) in float-float
// arithmetic on the FP32 pipes.
//
// GB300 runs FP64 at ~1 TFLOP/s but FP32 at ~72 TFLOP/s. A float-float number (hi, lo) carries 48
// significand bits; a float-float multiply-add costs ~11 FP32 operations (Dekker/Knuth: the product
// error by fma, TwoSum for the accumulation), which still gives ~6 TFLOP/s of 48-bit arithmetic.
// The whitening is one triangular matrix product of naux^2 * npair multiply-adds whose result already
// carries the metric's conditioning error (~kappa(L) eps_64), so 48 bits lose nothing measurable.
// Operands are converted once to (hi, lo) float pairs in place (same 8 bytes per element); the output
// is written in FP64 as hi + lo.
#include "common.cuh"

namespace dfhf {

namespace {

constexpr int BM = 128, BN = 128, BK = 8;
constexpr int NT = 256;   // 16 x 16 threads, 8 x 8 outputs each (rows ty + 16 i, columns tx + 16 j)

// x (double) -> (hi, lo) floats with hi + lo = x to ~2^-48 relative; in place over the same 8 bytes
__global__ void to_float_float_kernel(double* __restrict__ x, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    const float hi = (float)v;
    const float lo = (float)(v - (double)hi);
    reinterpret_cast<float2*>(x)[i] = make_float2(hi, lo);
}

__device__ __forceinline__ void df_fma(float& sh, float& sl, float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);       // exact rounding error of ah*bh
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float t = sh + p;           // TwoSum(sh, p)
    const float z = t - sh;
    const float err = (sh - (t - z)) + (p - z);
    sl += err + e;
    sh = t;
}

// C[m][n] = sum_{k <= m} L[m][k] A[k][n]; L (m x m, lower) and A (m x ncol, row stride ld) as float2
__global__ void __launch_bounds__(NT) trmm_ff_kernel(int m, long long ncol, const float2* __restrict__ L,
                                                     const float2* __restrict__ A, long long ld,
                                                     double* __restrict__ C) {
    __shared__ float2 As[2][BK][BM];
    __shared__ float2 Bs[2][BK][BN];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * BM;
    const long long n0 = (long long)blockIdx.x * BN;
    float sh[8][8], sl[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) sh[i][j] = sl[i][j] = 0.f;
    const int kend = min(m, m0 + BM);   // L is lower triangular
    // register staging: 4 L elements and 4 A elements per thread per k-tile
    float2 ra[4], rb[4];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = tid + q * NT;
            const int r = idx / BK, c = idx % BK;
            const int gm = m0 + r, gk = k0 + c;
            ra[q] = (gm < m && gk < m) ? L[(long long)gm * m + gk] : make_float2(0.f, 0.f);
            const int rr = idx / BN, cc = idx % BN;
            const int gk2 = k0 + rr;
            const long long gn = n0 + cc;
            rb[q] = (gk2 < m && gn < ncol) ? A[(long long)gk2 * ld + gn] : make_float2(0.f, 0.f);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = tid + q * NT;
            As[buf][idx % BK][idx / BK] = ra[q];
            Bs[buf][idx / BN][idx % BN] = rb[q];
        }
    };
    fetch(0);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < kend; k0 += BK) {
        const bool more = k0 + BK < kend;
        if (more) fetch(k0 + BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            float2 a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[buf][k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = Bs[buf][k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) df_fma(sh[i][j], sl[i][j], a[i].x, a[i].y, b[j].x, b[j].y);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= m) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const long long gn = n0 + tx + 16 * j;
            if (gn < ncol) C[(long long)gm * ld + gn] = (double)sh[i][j] + (double)sl[i][j];
        }
    }
}

// back to FP64 in place: x = hi + lo
__global__ void from_float_float_kernel(double* __restrict__ x, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 v = reinterpret_cast<const float2*>(x)[i];
    x[i] = (double)v.x + (double)v.y;
}

}  // namespace

// B = L^-1 A in float-float. Linv (m x m, FP64) is copied to Lff (m x m doubles of scratch) as float
// pairs; A (m x ncol FP64, row stride ld) is converted to float pairs in place and, if restore_a,
// back to FP64 afterwards (equal to the input to ~2^-48 relative). B receives FP64.
void whiten_float_float(cudaStream_t s, int m, long long ncol, const double* Linv, double* Lff, double* A, double* B,
                        long long ld, bool restore_a) {
    const long long nl = (long long)m * m, na = (long long)m * ld;
    DF_CUDA(cudaMemcpyAsync(Lff, Linv, sizeof(double) * nl, cudaMemcpyDeviceToDevice, s));
    to_float_float_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, s>>>(Lff, nl);
    DF_CHECK_LAUNCH();
    to_float_float_kernel<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(A, na);
    DF_CHECK_LAUNCH();
    const long long chunk = 65535LL * BN;
    for (long long c0 = 0; c0 < ncol; c0 += chunk) {
        const long long nc = (ncol - c0 < chunk) ? ncol - c0 : chunk;
        dim3 grid((unsigned)((nc + BN - 1) / BN), (m + BM - 1) / BM);
        trmm_ff_kernel<<<grid, NT, 0, s>>>(m, nc, reinterpret_cast<const float2*>(Lff),
                                           reinterpret_cast<const float2*>(A) + c0, ld, B + c0);
        DF_CHECK_LAUNCH();
    }
    if (restore_a) {
        from_float_float_kernel<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(A, na);
        DF_CHECK_LAUNCH();
    }
}

}  // namespace dfhf
