// Rys-quadrature evaluation of (c | a b) over uncontracted Cartesian Gaussians for one class.
//
// c: single Gaussian (exponent eta, centre C); a, b: bra pair (zeta = alpha_a + alpha_b, product
// centre Q, K_ab = exp(-alpha_a alpha_b |A-B|^2 / zeta)); rho = zeta eta/(zeta+eta),
// W = (zeta Q + eta C)/(zeta+eta), T = rho |Q-C|^2. With the N = floor(L/2)+1 Rys nodes u_r = t_r^2
// and weights w_r of T (rys.cuh), the integral factorises per root into 1-D integrals:
//   (c|a b) = pref * sum_r w_r I_x(p_x, a_x, b_x; u_r) I_y(...) I_z(...),
//   pref = 2 pi^{5/2} K_ab / (zeta eta sqrt(zeta+eta)).
// The 1-D integrals follow from the Obara-Saika vertical recurrences with [.]^(m+1) -> u [.]
// (Rys, Dupuis & King, J. Comput. Chem. 4, 154 (1983)):
//   I(e+1, p) = C00 I(e,p) + e B10 I(e-1,p) + p B00 I(e,p-1)
//   I(0, p+1) = D00 I(0,p) + p B01 I(0,p-1)
//   C00 = (Q-A) + (W-Q) u, D00 = (W-C) u, B00 = u / (2(zeta+eta)),
//   B10 = (1 - rho u / zeta) / (2 zeta), B01 = (1 - rho u / eta) / (2 eta),
// and the horizontal recurrence I(p, a, b+1) = I(p, a+1, b) + (A-B) I(p, a, b) moves quanta from A
// to B. The nuclear attraction <a|1/|r-C||b> is the eta -> infinity limit: rho = zeta, W = C,
// B00 = B01 = 0, pref = 2 pi K_ab / zeta, T = zeta |Q-C|^2.
#pragma once
#include "cart_sph.cuh"
#include "rys.cuh"

namespace dfhf {

struct RysParams {
    double QA[3], WQ[3], WC[3], AB[3];
    double i2z, rz;     // 1/(2 zeta), rho/zeta
    double i2e, re;     // 1/(2 eta), rho/eta
    double i2ze;        // 1/(2 (zeta + eta))
};

// cart[p][a][b] (levels LP, LA, LB) += sum over roots; x, w: nodes and weights (pref folded into w)
template <int LP, int LA, int LB>
__device__ __forceinline__ void rys_cart(const RysParams& q, const double* x, const double* w, double* cart) {
    constexpr int LE = LA + LB;
    constexpr int N = (LP + LE) / 2 + 1;
    constexpr int CP = ncart(LP), CA = ncart(LA), CB = ncart(LB);
#pragma unroll
    for (int c = 0; c < CP * CA * CB; ++c) cart[c] = 0.0;
#pragma unroll(LP + LE > 5 ? 1 : N)
    for (int r = 0; r < N; ++r) {
        const double u = x[r];
        const double B00 = u * q.i2ze;
        const double B10 = q.i2z * (1.0 - q.rz * u);
        const double B01 = q.i2e * (1.0 - q.re * u);
        double G[3][LP + 1][LA + 1][LB + 1];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double C00 = q.QA[d] + q.WQ[d] * u;
            const double D00 = q.WC[d] * u;
            double I[LE + 1][LP + 1];
            I[0][0] = (d == 2) ? w[r] : 1.0;
#pragma unroll
            for (int p = 0; p < LP; ++p) I[0][p + 1] = D00 * I[0][p] + (p > 0 ? p * B01 * I[0][p - 1] : 0.0);
#pragma unroll
            for (int e = 0; e < LE; ++e)
#pragma unroll
                for (int p = 0; p <= LP; ++p) {
                    double v = C00 * I[e][p];
                    if (e > 0) v += e * B10 * I[e - 1][p];
                    if (p > 0) v += p * B00 * I[e][p - 1];
                    I[e + 1][p] = v;
                }
            // horizontal recurrence in 1-D: H[b][e] for e <= LE - b
            double H[LB + 1][LE + 1];
#pragma unroll
            for (int p = 0; p <= LP; ++p) {
#pragma unroll
                for (int e = 0; e <= LE; ++e) H[0][e] = I[e][p];
#pragma unroll
                for (int b = 0; b < LB; ++b)
#pragma unroll
                    for (int e = 0; e < LE - b; ++e) H[b + 1][e] = H[b][e + 1] + q.AB[d] * H[b][e];
#pragma unroll
                for (int a = 0; a <= LA; ++a)
#pragma unroll
                    for (int b = 0; b <= LB; ++b) G[d][p][a][b] = H[b][a];
            }
        }
        // accumulate the Cartesian products
#pragma unroll
        for (int pi = LP; pi >= 0; --pi)
#pragma unroll
            for (int pj = LP - pi; pj >= 0; --pj) {
                const int pk = LP - pi - pj;
                const int ip = cidx(pj, pk);
#pragma unroll
                for (int ai = LA; ai >= 0; --ai)
#pragma unroll
                    for (int aj = LA - ai; aj >= 0; --aj) {
                        const int ak = LA - ai - aj;
                        const int ia = cidx(aj, ak);
#pragma unroll
                        for (int bi = LB; bi >= 0; --bi)
#pragma unroll
                            for (int bj = LB - bi; bj >= 0; --bj) {
                                const int bk = LB - bi - bj;
                                const int ib = cidx(bj, bk);
                                cart[(ip * CA + ia) * CB + ib] +=
                                    G[0][pi][ai][bi] * G[1][pj][aj][bj] * G[2][pk][ak][bk];
                            }
                    }
            }
    }
}

}  // namespace dfhf
