/*
 * ORACLE -- test infrastructure only. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg may load this library. The product path never calls it.
 *
 * Plain FP64 molecular integrals over uncontracted real-solid-harmonic Gaussian shells by the
 * McMurchie-Davidson scheme (Hermite expansion coefficients E^{ij}_t and Hermite Coulomb
 * integrals R^n_{tuv}); see Helgaker, Joergensen & Olsen, "Molecular Electronic-Structure
 * Theory" (2000), sections 9.5 (E coefficients), 9.9 (R integrals), 9.7-9.10 (S, T, V, ERI),
 * and eq. 6.4.47-6.4.48 / Table 6.3 (real solid harmonics).
 *
 * The paper (section "Molecular integrals") states that the two-electron integrals with the
 * 1/r12 kernel are evaluated by standard algorithms over shell objects, the nuclear attraction
 * needing the molecule as well. This file evaluates exactly those integrals by a scheme that is
 * deliberately different from the Obara-Saika recurrences of the CUDA path; the two share no code.
 *
 * Nothing here is blocked, fused or reordered for speed beyond looping over shells.
 *
 * Basis convention: function chi_{lm}(r) = N_l S_lm(r - A) exp(-alpha |r - A|^2) with S_lm the
 * real solid harmonics (Helgaker eq. 6.4.47), m ordered -l..l, N chosen numerically so that
 * <chi|chi> = 1 (computed here from this file's own overlap integral).
 * Cartesian order within a shell: x power descending, then y power descending.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_LMAX 4          /* shells up to g are accepted by the primitive routines */
#define OR_LSUM 12         /* largest total angular momentum (4 x l=3) */

/* ---------------------------------------------------------------------------------------------
 * Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt.
 * T <= 40: the convergent series F_m(T) = exp(-T) sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)),
 *          evaluated for the largest m, then the downward recursion
 *          F_m = (2T F_{m+1} + exp(-T)) / (2m+1).
 * T >  40: F_0 = sqrt(pi/T)/2 * erf(sqrt T) and the upward recursion
 *          F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T), stable for T >> m.
 * ------------------------------------------------------------------------------------------- */
void or_boys(int mmax, double T, double* F) {
    if (T <= 40.0) {
        double term = 1.0 / (2 * mmax + 1), sum = term;
        for (int k = 1; k < 2000; ++k) {
            term *= 2.0 * T / (2 * mmax + 2 * k + 1);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        double e = exp(-T);
        F[mmax] = e * sum;
        for (int m = mmax - 1; m >= 0; --m) F[m] = (2.0 * T * F[m + 1] + e) / (2 * m + 1);
    } else {
        double e = exp(-T);
        F[0] = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
        for (int m = 0; m < mmax; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0 * T);
    }
}

/* ---------------------------------------------------------------------------------------------
 * Hermite expansion coefficients (Helgaker eq. 9.5.6-9.5.7) for one Cartesian direction:
 * E[i][j][t] for i <= imax, j <= jmax, 0 <= t <= i + j.  a, b: exponents; Xab = A - B.
 * b = 0 gives the expansion of a single Gaussian (used for the auxiliary functions).
 * ------------------------------------------------------------------------------------------- */
#define EDIM (OR_LMAX + 3)
typedef double Etab[EDIM][EDIM][2 * EDIM + 1];

static void hermite_E(int imax, int jmax, double a, double b, double Xab, Etab E) {
    double p = a + b, mu = a * b / p;
    double Xpa = -b / p * Xab, Xpb = a / p * Xab;
    memset(E, 0, sizeof(Etab));
    E[0][0][0] = exp(-mu * Xab * Xab);
    for (int i = 0; i <= imax; ++i) {
        for (int j = 0; j <= jmax; ++j) {
            if (i == 0 && j == 0) continue;
            for (int t = 0; t <= i + j; ++t) {
                double v;
                if (i > 0) {
                    v = Xpa * E[i - 1][j][t];
                    if (t > 0) v += E[i - 1][j][t - 1] / (2 * p);
                    if (t + 1 <= i - 1 + j) v += (t + 1) * E[i - 1][j][t + 1];
                } else {
                    v = Xpb * E[i][j - 1][t];
                    if (t > 0) v += E[i][j - 1][t - 1] / (2 * p);
                    if (t + 1 <= i + j - 1) v += (t + 1) * E[i][j - 1][t + 1];
                }
                E[i][j][t] = v;
            }
        }
    }
}

/* ---------------------------------------------------------------------------------------------
 * Hermite Coulomb integrals R^0_{tuv}(alpha, X, Y, Z) for t+u+v <= L (Helgaker eq. 9.9.18-9.9.20):
 * R^n_{000} = (-2 alpha)^n F_n(alpha R^2); R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X R^{n+1}_{t,u,v},
 * and likewise for u (Y) and v (Z). Result R[t][u][v] for n = 0.
 * ------------------------------------------------------------------------------------------- */
#define RD (OR_LSUM + 1)
typedef double Rtab[RD][RD][RD];

static void hermite_R(int L, double alpha, double X, double Y, double Z, Rtab R0) {
    static __thread double Rn[RD][RD][RD][RD];
    double F[RD + 1];
    or_boys(L, alpha * (X * X + Y * Y + Z * Z), F);
    double f = 1.0;
    for (int n = 0; n <= L; ++n) { Rn[n][0][0][0] = f * F[n]; f *= -2.0 * alpha; }
    /* build levels of total order s = t+u+v from 1 to L; R^n needs n <= L - s */
    for (int s = 1; s <= L; ++s) {
        for (int n = 0; n <= L - s; ++n) {
            for (int t = 0; t <= s; ++t) {
                for (int u = 0; u <= s - t; ++u) {
                    int v = s - t - u;
                    double r;
                    if (t > 0) {
                        r = X * Rn[n + 1][t - 1][u][v];
                        if (t > 1) r += (t - 1) * Rn[n + 1][t - 2][u][v];
                    } else if (u > 0) {
                        r = Y * Rn[n + 1][t][u - 1][v];
                        if (u > 1) r += (u - 1) * Rn[n + 1][t][u - 2][v];
                    } else {
                        r = Z * Rn[n + 1][t][u][v - 1];
                        if (v > 1) r += (v - 1) * Rn[n + 1][t][u][v - 2];
                    }
                    Rn[n][t][u][v] = r;
                }
            }
        }
    }
    for (int t = 0; t <= L; ++t)
        for (int u = 0; u <= L - t; ++u)
            for (int v = 0; v <= L - t - u; ++v) R0[t][u][v] = Rn[0][t][u][v];
}

/* ---------------------------------------------------------------------------------------------
 * Primitive Cartesian integrals (unnormalised x^i y^j z^k exp(-a r^2) about each centre).
 * pw* arrays are the three Cartesian powers.
 * ------------------------------------------------------------------------------------------- */
static void gauss_product(double a, const double* A, double b, const double* B, double* P) {
    for (int k = 0; k < 3; ++k) P[k] = (a * A[k] + b * B[k]) / (a + b);
}

/* overlap <a|b> (Helgaker eq. 9.3.12 with 9.5.7) */
double or_prim_overlap(const int* pa, double a, const double* A, const int* pb, double b, const double* B) {
    double p = a + b, s = pow(M_PI / p, 1.5);
    for (int k = 0; k < 3; ++k) {
        Etab E;
        hermite_E(pa[k], pb[k], a, b, A[k] - B[k], E);
        s *= E[pa[k]][pb[k]][0];
    }
    return s;
}

/* 1-D overlap factor sqrt(pi/p) E^{ij}_0; j may be up to pb+2 for the kinetic integral */
static double ov1d(int i, int j, double a, double b, double Xab) {
    if (j < 0 || i < 0) return 0.0;
    Etab E;
    hermite_E(i, j, a, b, Xab, E);
    return E[i][j][0] * sqrt(M_PI / (a + b));
}

/* kinetic <a| -1/2 nabla^2 |b> via d^2/dx^2 acting on b (Helgaker eq. 9.3.22-9.3.24) */
double or_prim_kinetic(const int* pa, double a, const double* A, const int* pb, double b, const double* B) {
    double S[3], T[3];
    for (int k = 0; k < 3; ++k) {
        double X = A[k] - B[k];
        int i = pa[k], j = pb[k];
        S[k] = ov1d(i, j, a, b, X);
        double d2 = 4 * b * b * ov1d(i, j + 2, a, b, X) - 2 * b * (2 * j + 1) * ov1d(i, j, a, b, X);
        if (j >= 2) d2 += j * (j - 1) * ov1d(i, j - 2, a, b, X);
        T[k] = -0.5 * d2;
    }
    return T[0] * S[1] * S[2] + S[0] * T[1] * S[2] + S[0] * S[1] * T[2];
}

/* <a| 1/|r - C| |b> (Helgaker eq. 9.9.32), positive operator (no charge, no sign) */
double or_prim_potential(const int* pa, double a, const double* A, const int* pb, double b,
                         const double* B, const double* C) {
    double p = a + b, P[3];
    gauss_product(a, A, b, B, P);
    Etab Ex, Ey, Ez;
    hermite_E(pa[0], pb[0], a, b, A[0] - B[0], Ex);
    hermite_E(pa[1], pb[1], a, b, A[1] - B[1], Ey);
    hermite_E(pa[2], pb[2], a, b, A[2] - B[2], Ez);
    int L = pa[0] + pa[1] + pa[2] + pb[0] + pb[1] + pb[2];
    static __thread Rtab R;
    hermite_R(L, p, P[0] - C[0], P[1] - C[1], P[2] - C[2], R);
    double s = 0.0;
    for (int t = 0; t <= pa[0] + pb[0]; ++t)
        for (int u = 0; u <= pa[1] + pb[1]; ++u)
            for (int v = 0; v <= pa[2] + pb[2]; ++v)
                s += Ex[pa[0]][pb[0]][t] * Ey[pa[1]][pb[1]][u] * Ez[pa[2]][pb[2]][v] * R[t][u][v];
    return 2.0 * M_PI / p * s;
}

/* (ab|cd) with 1/r12 (Helgaker eq. 9.9.33); b or d with exponent 0 and power 0 reduce a pair
 * to a single Gaussian, which gives the two- and three-centre integrals. */
double or_prim_eri(const int* pa, double a, const double* A, const int* pb, double b, const double* B,
                   const int* pc, double c, const double* Cc, const int* pd, double d, const double* D) {
    double p = a + b, q = c + d, P[3], Q[3];
    gauss_product(a, A, b, B, P);
    gauss_product(c, Cc, d, D, Q);
    double alpha = p * q / (p + q);
    Etab Eab[3], Ecd[3];
    for (int k = 0; k < 3; ++k) {
        hermite_E(pa[k], pb[k], a, b, A[k] - B[k], Eab[k]);
        hermite_E(pc[k], pd[k], c, d, Cc[k] - D[k], Ecd[k]);
    }
    int Lab[3], Lcd[3], L = 0;
    for (int k = 0; k < 3; ++k) { Lab[k] = pa[k] + pb[k]; Lcd[k] = pc[k] + pd[k]; L += Lab[k] + Lcd[k]; }
    static __thread Rtab R;
    hermite_R(L, alpha, P[0] - Q[0], P[1] - Q[1], P[2] - Q[2], R);
    double s = 0.0;
    for (int t = 0; t <= Lab[0]; ++t)
        for (int u = 0; u <= Lab[1]; ++u)
            for (int v = 0; v <= Lab[2]; ++v) {
                double eab = Eab[0][pa[0]][pb[0]][t] * Eab[1][pa[1]][pb[1]][u] * Eab[2][pa[2]][pb[2]][v];
                if (eab == 0.0) continue;
                double inner = 0.0;
                for (int tau = 0; tau <= Lcd[0]; ++tau)
                    for (int nu = 0; nu <= Lcd[1]; ++nu)
                        for (int phi = 0; phi <= Lcd[2]; ++phi) {
                            double ecd = Ecd[0][pc[0]][pd[0]][tau] * Ecd[1][pc[1]][pd[1]][nu] *
                                         Ecd[2][pc[2]][pd[2]][phi];
                            double sg = ((tau + nu + phi) & 1) ? -1.0 : 1.0;
                            inner += sg * ecd * R[t + tau][u + nu][v + phi];
                        }
                s += eab * inner;
            }
    return 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q)) * s;
}

/* ---------------------------------------------------------------------------------------------
 * Real solid harmonics (Helgaker eq. 6.4.47-6.4.48):
 *   S_lm = N_lm sum_{t=0}^{(l-|m|)/2} sum_{u=0}^{t} sum_{v=v_m}^{floor(|m|/2 - v_m) + v_m}
 *          C^{lm}_{tuv} x^{2t+|m|-2(u+v)} y^{2(u+v)} z^{l-2t-|m|}
 *   C^{lm}_{tuv} = (-1)^{t+v-v_m} (1/4)^t binom(l,t) binom(l-t,|m|+t) binom(t,u) binom(|m|,2v)
 *   N_lm = (1/(2^|m| l!)) sqrt(2 (l+|m|)! (l-|m|)! / 2^{delta_m0}),  v_m = 0 (m >= 0), 1/2 (m < 0).
 * The sum over v runs over half-integers when m < 0 (v = 1/2, 3/2, ...): written with w = 2v.
 * Coefficient matrix cs[m + l][cart] over the Cartesian order described above.
 * ------------------------------------------------------------------------------------------- */
static double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}
static double fact(int n) { double r = 1.0; for (int i = 2; i <= n; ++i) r *= i; return r; }

int or_ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* index of Cartesian (i, j, k) with i + j + k = l in the x-descending, y-descending order */
static int cart_index(int l, int i, int j) {
    int before = 0;                     /* entries with a larger x power: sum_{i' > i} (l - i' + 1) */
    for (int ip = l; ip > i; --ip) before += l - ip + 1;
    return before + (l - i - j);
}

int or_cart_powers(int l, int* pw) {
    int n = 0;
    for (int i = l; i >= 0; --i)
        for (int j = l - i; j >= 0; --j) { pw[3 * n] = i; pw[3 * n + 1] = j; pw[3 * n + 2] = l - i - j; ++n; }
    return n;
}

void or_solid_harmonic_coeffs(int l, double* cs /* (2l+1) x ncart(l) */) {
    int nc = or_ncart(l);
    memset(cs, 0, sizeof(double) * (2 * l + 1) * nc);
    for (int m = -l; m <= l; ++m) {
        int am = abs(m);
        int twovm = (m < 0) ? 1 : 0;   /* 2 v_m */
        double Nlm = 1.0 / (pow(2.0, am) * fact(l)) *
                     sqrt(2.0 * fact(l + am) * fact(l - am) / (m == 0 ? 2.0 : 1.0));
        for (int t = 0; t <= (l - am) / 2; ++t)
            for (int u = 0; u <= t; ++u) {
                /* w = 2v runs over twovm, twovm + 2, ..., up to 2*floor(am/2 - vm) + twovm */
                int wmax = 2 * (int)floor(am / 2.0 - twovm / 2.0) + twovm;
                for (int w = twovm; w <= wmax; w += 2) {
                    int sgn_exp = t + (w - twovm) / 2;
                    double C = ((sgn_exp & 1) ? -1.0 : 1.0) * pow(0.25, t) * binom(l, t) *
                               binom(l - t, am + t) * binom(t, u) * binom(am, w);
                    /* x^{2t+|m|-2(u+v)} with 2v = w */
                    int px = 2 * t + am - 2 * u - w;
                    int py = 2 * u + w;
                    int pz = l - 2 * t - am;
                    if (px < 0 || py < 0 || pz < 0) continue;
                    cs[(m + l) * nc + cart_index(l, px, py)] += Nlm * C;
                }
            }
    }
}

/* ---------------------------------------------------------------------------------------------
 * Shell data and normalisation.
 * ------------------------------------------------------------------------------------------- */
typedef struct { int l; double a; double c[3]; } shell_t;

static void load_shells(int n, const int* l, const double* a, const double* xyz, shell_t* s) {
    for (int i = 0; i < n; ++i) { s[i].l = l[i]; s[i].a = a[i]; for (int k = 0; k < 3; ++k) s[i].c[k] = xyz[3 * i + k]; }
}

/* spherical normalisation: N^{-2} = sum_{cc'} cs_c cs_c' <c|c'> for m = 0 (all m share it) */
static double sph_norm(int l, double a) {
    int nc = or_ncart(l), pw[3 * 15];
    double cs[7 * 15], zero[3] = {0, 0, 0};
    or_cart_powers(l, pw);
    or_solid_harmonic_coeffs(l, cs);
    const double* row = cs + l * nc;   /* m = 0 */
    double s = 0.0;
    for (int i = 0; i < nc; ++i)
        for (int j = 0; j < nc; ++j)
            if (row[i] != 0.0 && row[j] != 0.0)
                s += row[i] * row[j] * or_prim_overlap(pw + 3 * i, a, zero, pw + 3 * j, a, zero);
    return 1.0 / sqrt(s);
}

/* normalisation of every m component separately (exported so a test can check they agree) */
void or_sph_norms(int l, double a, double* out /* 2l+1 */) {
    int nc = or_ncart(l), pw[3 * 15];
    double cs[7 * 15], zero[3] = {0, 0, 0};
    or_cart_powers(l, pw);
    or_solid_harmonic_coeffs(l, cs);
    for (int m = 0; m < 2 * l + 1; ++m) {
        const double* row = cs + m * nc;
        double s = 0.0;
        for (int i = 0; i < nc; ++i)
            for (int j = 0; j < nc; ++j)
                s += row[i] * row[j] * or_prim_overlap(pw + 3 * i, a, zero, pw + 3 * j, a, zero);
        out[m] = 1.0 / sqrt(s);
    }
}

static int offsets(int n, const shell_t* s, int* off) {
    int o = 0;
    for (int i = 0; i < n; ++i) { off[i] = o; o += 2 * s[i].l + 1; }
    return o;
}

/* ---------------------------------------------------------------------------------------------
 * Spherical shell blocks: transform a Cartesian block over up to four shells to normalised
 * spherical functions, one index at a time.
 * ------------------------------------------------------------------------------------------- */
static void sph_block2(const shell_t* A, const shell_t* B, double (*prim)(const int*, double, const double*,
                       const int*, double, const double*, const void*), const void* ctx, double* out) {
    int la = A->l, lb = B->l, nca = or_ncart(la), ncb = or_ncart(lb);
    int pa[45], pb[45];
    double ca[7 * 15], cb[7 * 15], cart[15 * 15], half[7 * 15];
    or_cart_powers(la, pa); or_cart_powers(lb, pb);
    or_solid_harmonic_coeffs(la, ca); or_solid_harmonic_coeffs(lb, cb);
    for (int i = 0; i < nca; ++i)
        for (int j = 0; j < ncb; ++j) cart[i * ncb + j] = prim(pa + 3 * i, A->a, A->c, pb + 3 * j, B->a, B->c, ctx);
    int nsa = 2 * la + 1, nsb = 2 * lb + 1;
    for (int ma = 0; ma < nsa; ++ma)
        for (int j = 0; j < ncb; ++j) {
            double s = 0.0;
            for (int i = 0; i < nca; ++i) s += ca[ma * nca + i] * cart[i * ncb + j];
            half[ma * ncb + j] = s;
        }
    double na = sph_norm(la, A->a), nb = sph_norm(lb, B->a);
    for (int ma = 0; ma < nsa; ++ma)
        for (int mb = 0; mb < nsb; ++mb) {
            double s = 0.0;
            for (int j = 0; j < ncb; ++j) s += half[ma * ncb + j] * cb[mb * ncb + j];
            out[ma * nsb + mb] = na * nb * s;
        }
}

static double prim_S(const int* pa, double a, const double* A, const int* pb, double b, const double* B, const void* c) {
    (void)c; return or_prim_overlap(pa, a, A, pb, b, B);
}
static double prim_T(const int* pa, double a, const double* A, const int* pb, double b, const double* B, const void* c) {
    (void)c; return or_prim_kinetic(pa, a, A, pb, b, B);
}
typedef struct { int natom; const double* Z; const double* R; } nuc_ctx;
static double prim_V(const int* pa, double a, const double* A, const int* pb, double b, const double* B, const void* c) {
    const nuc_ctx* nc = (const nuc_ctx*)c;
    double s = 0.0;
    for (int k = 0; k < nc->natom; ++k) s -= nc->Z[k] * or_prim_potential(pa, a, A, pb, b, B, nc->R + 3 * k);
    return s;
}
static const int ZP[3] = {0, 0, 0};
static double prim_2c(const int* pa, double a, const double* A, const int* pb, double b, const double* B, const void* c) {
    (void)c; return or_prim_eri(pa, a, A, ZP, 0.0, A, pb, b, B, ZP, 0.0, B);
}

/* which: 0 = overlap, 1 = kinetic, 2 = nuclear attraction (needs natom, Z, R) */
static void one_body(int which, int nsh, const int* l, const double* a, const double* xyz,
                     int natom, const double* Z, const double* R, double* out) {
    shell_t* s = (shell_t*)malloc(sizeof(shell_t) * nsh);
    int* off = (int*)malloc(sizeof(int) * nsh);
    load_shells(nsh, l, a, xyz, s);
    int n = offsets(nsh, s, off);
    nuc_ctx nc = {natom, Z, R};
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < nsh; ++i) {
        double blk[49];
        for (int j = 0; j < nsh; ++j) {
            if (which == 0) sph_block2(&s[i], &s[j], prim_S, NULL, blk);
            else if (which == 1) sph_block2(&s[i], &s[j], prim_T, NULL, blk);
            else if (which == 2) sph_block2(&s[i], &s[j], prim_V, &nc, blk);
            else sph_block2(&s[i], &s[j], prim_2c, NULL, blk);
            int ni = 2 * s[i].l + 1, nj = 2 * s[j].l + 1;
            for (int p = 0; p < ni; ++p)
                for (int q = 0; q < nj; ++q) out[(size_t)(off[i] + p) * n + off[j] + q] = blk[p * nj + q];
        }
    }
    free(s); free(off);
}

void or_overlap(int nsh, const int* l, const double* a, const double* xyz, double* out) {
    one_body(0, nsh, l, a, xyz, 0, NULL, NULL, out);
}
void or_kinetic(int nsh, const int* l, const double* a, const double* xyz, double* out) {
    one_body(1, nsh, l, a, xyz, 0, NULL, NULL, out);
}
void or_nuclear(int nsh, const int* l, const double* a, const double* xyz, int natom, const double* Z,
                const double* R, double* out) {
    one_body(2, nsh, l, a, xyz, natom, Z, R, out);
}
/* two-centre Coulomb metric (P|Q) over auxiliary shells */
void or_metric(int nsh, const int* l, const double* a, const double* xyz, double* out) {
    one_body(3, nsh, l, a, xyz, 0, NULL, NULL, out);
}

/* three-centre block (P|mu nu) for aux shell P and orbital shells M, N -> out[p][m][n] */
static void three_center_block(const shell_t* P, const shell_t* M, const shell_t* N, double* out) {
    int lp = P->l, lm = M->l, ln = N->l;
    int ncp = or_ncart(lp), ncm = or_ncart(lm), ncn = or_ncart(ln);
    int pp[45], pm[45], pn[45];
    double cp[7 * 15], cm[7 * 15], cn[7 * 15];
    or_cart_powers(lp, pp); or_cart_powers(lm, pm); or_cart_powers(ln, pn);
    or_solid_harmonic_coeffs(lp, cp); or_solid_harmonic_coeffs(lm, cm); or_solid_harmonic_coeffs(ln, cn);
    double* cart = (double*)malloc(sizeof(double) * ncp * ncm * ncn);
    for (int i = 0; i < ncp; ++i)
        for (int j = 0; j < ncm; ++j)
            for (int k = 0; k < ncn; ++k)
                cart[(i * ncm + j) * ncn + k] =
                    or_prim_eri(pp + 3 * i, P->a, P->c, ZP, 0.0, P->c, pm + 3 * j, M->a, M->c, pn + 3 * k, N->a, N->c);
    int nsp = 2 * lp + 1, nsm = 2 * lm + 1, nsn = 2 * ln + 1;
    double* t1 = (double*)malloc(sizeof(double) * nsp * ncm * ncn);
    double* t2 = (double*)malloc(sizeof(double) * nsp * nsm * ncn);
    for (int a = 0; a < nsp; ++a)
        for (int jk = 0; jk < ncm * ncn; ++jk) {
            double s = 0.0;
            for (int i = 0; i < ncp; ++i) s += cp[a * ncp + i] * cart[i * ncm * ncn + jk];
            t1[a * ncm * ncn + jk] = s;
        }
    for (int a = 0; a < nsp; ++a)
        for (int b = 0; b < nsm; ++b)
            for (int k = 0; k < ncn; ++k) {
                double s = 0.0;
                for (int j = 0; j < ncm; ++j) s += cm[b * ncm + j] * t1[(a * ncm + j) * ncn + k];
                t2[(a * nsm + b) * ncn + k] = s;
            }
    double np_ = sph_norm(lp, P->a), nm = sph_norm(lm, M->a), nn = sph_norm(ln, N->a);
    for (int a = 0; a < nsp; ++a)
        for (int b = 0; b < nsm; ++b)
            for (int c = 0; c < nsn; ++c) {
                double s = 0.0;
                for (int k = 0; k < ncn; ++k) s += cn[c * ncn + k] * t2[(a * nsm + b) * ncn + k];
                out[(a * nsm + b) * nsn + c] = np_ * nm * nn * s;
            }
    free(cart); free(t1); free(t2);
}

/* full three-centre tensor out[P][mu][nu] (naux x n x n) */
void or_three_center(int nsa, const int* la, const double* aa, const double* xa,
                     int nsh, const int* l, const double* a, const double* xyz, double* out) {
    shell_t* sa = (shell_t*)malloc(sizeof(shell_t) * nsa);
    shell_t* s = (shell_t*)malloc(sizeof(shell_t) * nsh);
    int* offa = (int*)malloc(sizeof(int) * nsa);
    int* off = (int*)malloc(sizeof(int) * nsh);
    load_shells(nsa, la, aa, xa, sa);
    load_shells(nsh, l, a, xyz, s);
    offsets(nsa, sa, offa);
    int n = offsets(nsh, s, off);
#pragma omp parallel for schedule(dynamic)
    for (int P = 0; P < nsa; ++P) {
        double blk[7 * 5 * 5 * 9];
        for (int M = 0; M < nsh; ++M)
            for (int N = 0; N <= M; ++N) {
                three_center_block(&sa[P], &s[M], &s[N], blk);
                int np_ = 2 * sa[P].l + 1, nm = 2 * s[M].l + 1, nn = 2 * s[N].l + 1;
                for (int p = 0; p < np_; ++p)
                    for (int i = 0; i < nm; ++i)
                        for (int j = 0; j < nn; ++j) {
                            double v = blk[(p * nm + i) * nn + j];
                            size_t base = (size_t)(offa[P] + p) * n * n;
                            out[base + (size_t)(off[M] + i) * n + off[N] + j] = v;
                            out[base + (size_t)(off[N] + j) * n + off[M] + i] = v;
                        }
            }
    }
    free(sa); free(s); free(offa); free(off);
}

/* selected shell triples (P, M, N): blocks [p][m][n] concatenated in list order */
void or_three_center_triples(int nsa, const int* la, const double* aa, const double* xa,
                             int nsh, const int* l, const double* a, const double* xyz,
                             int ntrip, const int* trip, const long* out_off, double* out) {
    shell_t* sa = (shell_t*)malloc(sizeof(shell_t) * nsa);
    shell_t* s = (shell_t*)malloc(sizeof(shell_t) * nsh);
    load_shells(nsa, la, aa, xa, sa);
    load_shells(nsh, l, a, xyz, s);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < ntrip; ++t)
        three_center_block(&sa[trip[3 * t]], &s[trip[3 * t + 1]], &s[trip[3 * t + 2]], out + out_off[t]);
    free(sa); free(s);
}

/* conventional four-index (mu nu|la si) over spherical functions, out[n^4]; tiny systems only.
 * Each shell quartet: Cartesian block, then the spherical transform one index at a time. */
static void sph_transform_index(const double* in, double* out, int pre, int nc, int ns, int post, const double* cs) {
    for (int a = 0; a < pre; ++a)
        for (int m = 0; m < ns; ++m)
            for (int b = 0; b < post; ++b) {
                double s = 0.0;
                for (int c = 0; c < nc; ++c) s += cs[m * nc + c] * in[((size_t)a * nc + c) * post + b];
                out[((size_t)a * ns + m) * post + b] = s;
            }
}

void or_four_center(int nsh, const int* l, const double* a, const double* xyz, double* out) {
    shell_t* s = (shell_t*)malloc(sizeof(shell_t) * nsh);
    int* off = (int*)malloc(sizeof(int) * nsh);
    load_shells(nsh, l, a, xyz, s);
    int n = offsets(nsh, s, off);
#pragma omp parallel for schedule(dynamic) collapse(2)
    for (int A = 0; A < nsh; ++A)
        for (int B = 0; B < nsh; ++B) {
            double* buf0 = (double*)malloc(sizeof(double) * 15 * 15 * 15 * 15);
            double* buf1 = (double*)malloc(sizeof(double) * 15 * 15 * 15 * 15);
            for (int C = 0; C < nsh; ++C)
                for (int D = 0; D < nsh; ++D) {
                    const shell_t* S4[4] = {&s[A], &s[B], &s[C], &s[D]};
                    int nc[4], ns[4], pw[4][45];
                    double cs[4][7 * 15], nrm = 1.0;
                    for (int k = 0; k < 4; ++k) {
                        nc[k] = or_ncart(S4[k]->l); ns[k] = 2 * S4[k]->l + 1;
                        or_cart_powers(S4[k]->l, pw[k]); or_solid_harmonic_coeffs(S4[k]->l, cs[k]);
                        nrm *= sph_norm(S4[k]->l, S4[k]->a);
                    }
                    for (int i = 0; i < nc[0]; ++i)
                        for (int j = 0; j < nc[1]; ++j)
                            for (int k = 0; k < nc[2]; ++k)
                                for (int m = 0; m < nc[3]; ++m)
                                    buf0[((i * nc[1] + j) * nc[2] + k) * nc[3] + m] =
                                        or_prim_eri(pw[0] + 3 * i, S4[0]->a, S4[0]->c, pw[1] + 3 * j, S4[1]->a, S4[1]->c,
                                                    pw[2] + 3 * k, S4[2]->a, S4[2]->c, pw[3] + 3 * m, S4[3]->a, S4[3]->c);
                    /* index 0 */
                    sph_transform_index(buf0, buf1, 1, nc[0], ns[0], nc[1] * nc[2] * nc[3], cs[0]);
                    sph_transform_index(buf1, buf0, ns[0], nc[1], ns[1], nc[2] * nc[3], cs[1]);
                    sph_transform_index(buf0, buf1, ns[0] * ns[1], nc[2], ns[2], nc[3], cs[2]);
                    sph_transform_index(buf1, buf0, ns[0] * ns[1] * ns[2], nc[3], ns[3], 1, cs[3]);
                    for (int i = 0; i < ns[0]; ++i)
                        for (int j = 0; j < ns[1]; ++j)
                            for (int k = 0; k < ns[2]; ++k)
                                for (int m = 0; m < ns[3]; ++m) {
                                    size_t idx = (((size_t)(off[A] + i) * n + off[B] + j) * n + off[C] + k) * n + off[D] + m;
                                    out[idx] = nrm * buf0[((i * ns[1] + j) * ns[2] + k) * ns[3] + m];
                                }
                }
            free(buf0); free(buf1);
        }
    free(s); free(off);
}
