// Cartesian Gaussian component ordering and the Cartesian -> real-solid-harmonic transformation.
//
// Cartesian components of total l are ordered x^l first, then by descending y power; the index of
// x^i y^j z^k within its level is (j+k)(j+k+1)/2 + k.
#pragma once
#include <cuda_runtime.h>

namespace dfhf {

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
__host__ __device__ constexpr int ncum(int l) { return l * (l + 1) * (l + 2) / 6; }
__host__ __device__ constexpr int cidx(int j, int k) { return (j + k) * (j + k + 1) / 2 + k; }
__host__ __device__ constexpr int nsph(int l) { return 2 * l + 1; }

// ------------------------------------------------------------------------------------------------
// Cartesian -> real solid harmonics (m = -l..l), along one index with strides; coefficients of the
// standard real solid harmonics (Helgaker, Joergensen & Olsen, Molecular Electronic-Structure Theory,
// Table 6.3): l=1: y, z, x;  l=2: sqrt3 xy, sqrt3 yz, z^2 - (x^2+y^2)/2, sqrt3 xz, sqrt3/2 (x^2-y^2);
// l=3: sqrt(5/8)(3x^2 y - y^3), sqrt15 xyz, sqrt(3/8) y(4z^2-x^2-y^2), z(2z^2-3x^2-3y^2)/2,
//      sqrt(3/8) x(4z^2-x^2-y^2), sqrt15/2 z(x^2-y^2), sqrt(5/8)(x^3 - 3xy^2).
// ------------------------------------------------------------------------------------------------
template <int L>
struct Sph;

template <>
struct Sph<0> {
    template <int IS, int OS>
    __device__ __forceinline__ static void apply(const double* in, double* out) { out[0] = in[0]; }
};
template <>
struct Sph<1> {
    template <int IS, int OS>
    __device__ __forceinline__ static void apply(const double* in, double* out) {
        out[0] = in[1 * IS];
        out[OS] = in[2 * IS];
        out[2 * OS] = in[0];
    }
};
template <>
struct Sph<2> {
    template <int IS, int OS>
    __device__ __forceinline__ static void apply(const double* in, double* out) {
        constexpr double s3 = 1.7320508075688772935, hs3 = 0.86602540378443864676;
        // cart: 0 xx, 1 xy, 2 xz, 3 yy, 4 yz, 5 zz
        out[0] = s3 * in[1 * IS];
        out[OS] = s3 * in[4 * IS];
        out[2 * OS] = in[5 * IS] - 0.5 * (in[0] + in[3 * IS]);
        out[3 * OS] = s3 * in[2 * IS];
        out[4 * OS] = hs3 * (in[0] - in[3 * IS]);
    }
};
template <>
struct Sph<3> {
    template <int IS, int OS>
    __device__ __forceinline__ static void apply(const double* in, double* out) {
        constexpr double c58 = 0.79056941504209483300;   // sqrt(5/8)
        constexpr double c15 = 3.8729833462074168852;    // sqrt(15)
        constexpr double c38 = 0.61237243569579452455;   // sqrt(3/8)
        // cart: 0 xxx, 1 xxy, 2 xxz, 3 xyy, 4 xyz, 5 xzz, 6 yyy, 7 yyz, 8 yzz, 9 zzz
        out[0] = c58 * (3.0 * in[1 * IS] - in[6 * IS]);
        out[OS] = c15 * in[4 * IS];
        out[2 * OS] = c38 * (4.0 * in[8 * IS] - in[1 * IS] - in[6 * IS]);
        out[3 * OS] = in[9 * IS] - 1.5 * (in[2 * IS] + in[7 * IS]);
        out[4 * OS] = c38 * (4.0 * in[5 * IS] - in[0] - in[3 * IS]);
        out[5 * OS] = 0.5 * c15 * (in[2 * IS] - in[7 * IS]);
        out[6 * OS] = c58 * (in[0] - 3.0 * in[3 * IS]);
    }
};

// cart[p][a][b] -> sph[mp][ma][mb]
template <int LP, int LA, int LB>
__device__ __forceinline__ void cart_to_sph(const double* cart, double* sph) {
    constexpr int CP = ncart(LP), CA = ncart(LA), CB = ncart(LB);
    constexpr int SP = nsph(LP), SA = nsph(LA), SB = nsph(LB);
    double t1[CP * CA * SB];
#pragma unroll
    for (int pa = 0; pa < CP * CA; ++pa) Sph<LB>::template apply<1, 1>(cart + pa * CB, t1 + pa * SB);
    double t2[CP * SA * SB];
#pragma unroll
    for (int p = 0; p < CP; ++p)
#pragma unroll
        for (int b = 0; b < SB; ++b)
            Sph<LA>::template apply<SB, SB>(t1 + p * CA * SB + b, t2 + p * SA * SB + b);
#pragma unroll
    for (int ab = 0; ab < SA * SB; ++ab) Sph<LP>::template apply<SA * SB, SA * SB>(t2 + ab, sph + ab);
}

}  // namespace dfhf
