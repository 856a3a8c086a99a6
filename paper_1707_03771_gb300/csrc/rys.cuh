// Rys quadrature roots and weights (paper, section "Molecular integrals": electron-repulsion
// integrals by the Rys-quadrature algorithm, Dupuis, Rys & King, J. Chem. Phys. 65, 111 (1976)).
//
// For n roots, nodes x_i = t_i^2 in (0,1) and weights w_i reproduce the Boys function moments
//     sum_i w_i x_i^k = F_k(T) = int_0^1 t^{2k} exp(-T t^2) dt,   k = 0 .. 2n-1,
// i.e. they are the Gauss rule of the measure exp(-T x) x^{-1/2} dx / 2 on [0,1].
// T < 60: piecewise Chebyshev interpolation (degree RYS_DEG on unit intervals of T) of nodes and
//         weights tabulated on the host (rys_table.cu: discretised Stieltjes procedure + Jacobi
//         matrix eigen-decomposition in long double).
// T >= 60: the measure differs from exp(-T x) x^{-1/2} dx / 2 on [0, inf) by < 1e-17 relative,
//         whose Gauss rule is generalised Gauss-Laguerre (alpha = -1/2) scaled: x_i = r_i / T,
//         w_i = W_i / (2 sqrt T).
#pragma once
#include <cuda_runtime.h>

namespace dfhf {

constexpr int RYS_NMAX = 4;
constexpr int RYS_DEG = 15;                 // Chebyshev degree per interval
constexpr int RYS_NC = RYS_DEG + 1;
constexpr int RYS_NINT = 60;                // unit intervals [k, k+1), k = 0..59
constexpr double RYS_TMAX = 60.0;

__host__ __device__ constexpr int rys_offset(int n) {   // start of the n-root block (n >= 1)
    return RYS_NINT * RYS_NC * (n - 1) * n;             // sum_{m<n} 2m * NINT * NC
}
constexpr int RYS_ASYM = rys_offset(RYS_NMAX + 1);      // Laguerre nodes/weights: n*(n-1)/2 .. per n
constexpr int RYS_TABLE_SIZE = RYS_ASYM + 2 * (RYS_NMAX * (RYS_NMAX + 1) / 2);

__host__ __device__ inline double chebyshev_eval(const double* c, double s) {
    double b1 = 0.0, b2 = 0.0;
    const double s2 = 2.0 * s;
    for (int k = RYS_DEG; k >= 1; --k) {
        const double b0 = c[k] + s2 * b1 - b2;
        b2 = b1;
        b1 = b0;
    }
    return c[0] + s * b1 - b2;
}

template <int N>
__host__ __device__ inline void rys_roots(double T, const double* __restrict__ tab, double* x, double* w) {
    if (T < RYS_TMAX) {
        const int k = (int)T;
        const double s = 2.0 * (T - k) - 1.0;
        const double* c = tab + rys_offset(N) + k * (2 * N) * RYS_NC;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            x[i] = chebyshev_eval(c + i * RYS_NC, s);
            w[i] = chebyshev_eval(c + (N + i) * RYS_NC, s);
        }
    } else {
        const double inv = 1.0 / T;
        const double sq = sqrt(inv);
        const double* a = tab + RYS_ASYM + N * (N - 1);   // N nodes then N half-weights
#pragma unroll
        for (int i = 0; i < N; ++i) {
            x[i] = a[i] * inv;
            w[i] = a[N + i] * sq;
        }
    }
}

const double* rys_table_device();
const double* rys_table_host();

}  // namespace dfhf
