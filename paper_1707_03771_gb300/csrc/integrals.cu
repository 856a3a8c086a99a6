// Integral kernels: three-centre (P|mu nu) (the integral hot loop), the two-centre Coulomb metric
// (P|Q), and the one-electron overlap, kinetic and nuclear-attraction matrices.
//
// Paper, section "Molecular integrals": the 1/r12 integrals are computed by Rys quadrature over shell
// objects, and the nuclear attraction needs the molecule as well. One kernel is instantiated per
// angular-momentum class; one thread evaluates one shell triple (or shell pair) with rys_eri.cuh.
#include <cmath>

#include "common.cuh"
#include "rys_eri.cuh"

namespace dfhf {

namespace {

constexpr double PI = 3.14159265358979323846;
constexpr double TWO_PI_52 = 34.986836655249725693;   // 2 pi^{5/2}

struct ShellView {
    const int* __restrict__ l;
    const int* __restrict__ off;
    const double* __restrict__ alpha;
    const double* __restrict__ norm;
    const double* __restrict__ xyz;
};
ShellView view(const ShellTable& t) { return {t.l, t.off, t.alpha, t.norm, t.xyz}; }

// bra pair (a, b) and ket single Gaussian c -> Rys nodes, weights (prefactor folded in), parameters
template <int N>
__device__ __forceinline__ void setup_3c(double aa, const double* A, double ab, const double* B, double eta,
                                         const double* C, const double* __restrict__ tab, RysParams& q,
                                         double* x, double* w) {
    const double zeta = aa + ab;
    const double iz = 1.0 / zeta;
    double Q[3], AB2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        Q[d] = (aa * A[d] + ab * B[d]) * iz;
        q.AB[d] = A[d] - B[d];
        AB2 += q.AB[d] * q.AB[d];
    }
    const double Kab = exp(-aa * ab * iz * AB2);
    const double ize = 1.0 / (zeta + eta);
    const double rho = zeta * eta * ize;
    double QC2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double W = (zeta * Q[d] + eta * C[d]) * ize;
        q.QA[d] = Q[d] - A[d];
        q.WQ[d] = W - Q[d];
        q.WC[d] = W - C[d];
        QC2 += (Q[d] - C[d]) * (Q[d] - C[d]);
    }
    const double ie = 1.0 / eta;
    q.i2z = 0.5 * iz;
    q.rz = rho * iz;
    q.i2e = 0.5 * ie;
    q.re = rho * ie;
    q.i2ze = 0.5 * ize;
    rys_roots<N>(rho * QC2, tab, x, w);
    const double pref = TWO_PI_52 * iz * ie * sqrt(ize) * Kab;
#pragma unroll
    for (int r = 0; r < N; ++r) w[r] *= pref;
}

template <int L>
struct NR {
    static constexpr int value = L / 2 + 1;
};

__device__ __forceinline__ void load3(const double* __restrict__ xyz, int s, double* c) {
    c[0] = xyz[3 * s];
    c[1] = xyz[3 * s + 1];
    c[2] = xyz[3 * s + 2];
}

// ---------------------------------------------------------------------------------------------
// three-centre (P|ab): threads over orbital shell pairs of one class, blockIdx.y over auxiliary
// shells of angular momentum LP; output rows of `row` doubles, packed mu >= nu tiles
// ---------------------------------------------------------------------------------------------
template <int LP, int LA, int LB>
__global__ void __launch_bounds__(128) eri3c_kernel(ShellView bas, ShellView aux, const int2* __restrict__ pairs,
                                                    int npairs, const int* __restrict__ auxl, int naux_l,
                                                    const double* __restrict__ tab, double* __restrict__ out,
                                                    long long row) {
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npairs) return;
    const int2 pr = pairs[ip];
    const int a = pr.x, b = pr.y;
    double A[3], B[3];
    load3(bas.xyz, a, A);
    load3(bas.xyz, b, B);
    const double aa = bas.alpha[a], ab = bas.alpha[b];
    const double nab = bas.norm[a] * bas.norm[b];
    const int offa = bas.off[a], offb = bas.off[b];
    for (int ia = blockIdx.y; ia < naux_l; ia += gridDim.y) {
        const int P = auxl[ia];
        double C[3];
        load3(aux.xyz, P, C);
        RysParams q;
        constexpr int N = NR<LP + LA + LB>::value;
        double x[N], w[N];
        setup_3c<N>(aa, A, ab, B, aux.alpha[P], C, tab, q, x, w);
        double cart[ncart(LP) * ncart(LA) * ncart(LB)];
        rys_cart<LP, LA, LB>(q, x, w, cart);
        double sph[nsph(LP) * nsph(LA) * nsph(LB)];
        cart_to_sph<LP, LA, LB>(cart, sph);
        const double scale = nab * aux.norm[P];
        const int offp = aux.off[P];
#pragma unroll
        for (int mp = 0; mp < nsph(LP); ++mp) {
            double* o = out + (long long)(offp + mp) * row;
#pragma unroll
            for (int ma = 0; ma < nsph(LA); ++ma)
#pragma unroll
                for (int mb = 0; mb < nsph(LB); ++mb) {
                    const int mu = offa + ma, nu = offb + mb;
                    const double v = scale * sph[(mp * nsph(LA) + ma) * nsph(LB) + mb];
                    o[packed_index(mu, nu)] = v;
                    if (mu / TS == nu / TS) o[packed_index(nu, mu)] = v;
                }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// two-centre metric (X|Y): X plays the single Gaussian, Y the bra with a null partner (exponent 0)
// ---------------------------------------------------------------------------------------------
template <int LX, int LY>
__global__ void __launch_bounds__(128) metric_kernel(ShellView aux, const int2* __restrict__ pairs, int npairs,
                                                     const double* __restrict__ tab, double* __restrict__ V,
                                                     int naux) {
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npairs) return;
    const int2 pr = pairs[ip];
    const int x = pr.x, y = pr.y;
    double X[3], Y[3];
    load3(aux.xyz, x, X);
    load3(aux.xyz, y, Y);
    RysParams q;
    constexpr int N = NR<LX + LY>::value;
    double xr[N], wr[N];
    setup_3c<N>(aux.alpha[y], Y, 0.0, Y, aux.alpha[x], X, tab, q, xr, wr);
    double cart[ncart(LX) * ncart(LY)];
    rys_cart<LX, LY, 0>(q, xr, wr, cart);
    double sph[nsph(LX) * nsph(LY)];
    cart_to_sph<LX, LY, 0>(cart, sph);
    const double scale = aux.norm[x] * aux.norm[y];
    const int ox = aux.off[x], oy = aux.off[y];
#pragma unroll
    for (int i = 0; i < nsph(LX); ++i)
#pragma unroll
        for (int j = 0; j < nsph(LY); ++j) {
            const double v = scale * sph[i * nsph(LY) + j];
            V[(long long)(ox + i) * naux + oy + j] = v;
            V[(long long)(oy + j) * naux + ox + i] = v;
        }
}

// ---------------------------------------------------------------------------------------------
// nuclear attraction: sum over nuclei of -Z <a|1/|r-C||b>
// ---------------------------------------------------------------------------------------------
template <int LA, int LB>
__global__ void __launch_bounds__(128) nuclear_kernel(ShellView bas, const int2* __restrict__ pairs, int npairs,
                                                      const double* __restrict__ axyz, const double* __restrict__ aZ,
                                                      int natom, const double* __restrict__ tab,
                                                      double* __restrict__ Vm, int n) {
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npairs) return;
    const int2 pr = pairs[ip];
    const int a = pr.x, b = pr.y;
    double A[3], B[3];
    load3(bas.xyz, a, A);
    load3(bas.xyz, b, B);
    const double aa = bas.alpha[a], ab = bas.alpha[b];
    const double zeta = aa + ab, iz = 1.0 / zeta;
    double Q[3], AB2 = 0.0;
    RysParams q;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        Q[d] = (aa * A[d] + ab * B[d]) * iz;
        q.AB[d] = A[d] - B[d];
        AB2 += q.AB[d] * q.AB[d];
        q.QA[d] = Q[d] - A[d];
        q.WC[d] = 0.0;
    }
    q.i2z = 0.5 * iz;
    q.rz = 1.0;
    q.i2e = q.re = q.i2ze = 0.0;
    const double base = 2.0 * PI * iz * exp(-aa * ab * iz * AB2);
    constexpr int NC = ncart(LA) * ncart(LB);
    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    for (int at = 0; at < natom; ++at) {
        double C[3] = {axyz[3 * at], axyz[3 * at + 1], axyz[3 * at + 2]};
        double QC2 = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            q.WQ[d] = C[d] - Q[d];
            QC2 += (Q[d] - C[d]) * (Q[d] - C[d]);
        }
        constexpr int N = NR<LA + LB>::value;
        double xr[N], wr[N];
        rys_roots<N>(zeta * QC2, tab, xr, wr);
        const double pref = -aZ[at] * base;
#pragma unroll
        for (int r = 0; r < N; ++r) wr[r] *= pref;
        double cart[NC];
        rys_cart<0, LA, LB>(q, xr, wr, cart);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] += cart[c];
    }
    double sph[nsph(LA) * nsph(LB)];
    cart_to_sph<0, LA, LB>(acc, sph);
    const double scale = bas.norm[a] * bas.norm[b];
    const int oa = bas.off[a], ob = bas.off[b];
#pragma unroll
    for (int i = 0; i < nsph(LA); ++i)
#pragma unroll
        for (int j = 0; j < nsph(LB); ++j) {
            const double v = scale * sph[i * nsph(LB) + j];
            Vm[(long long)(oa + i) * n + ob + j] = v;
            Vm[(long long)(ob + j) * n + oa + i] = v;
        }
}

// ---------------------------------------------------------------------------------------------
// overlap and kinetic: 1-D Obara-Saika overlap recurrences per direction,
//   S_{i+1,j} = (Q-A) S_ij + (i S_{i-1,j} + j S_{i,j-1}) / (2 zeta)
//   S_{i,j+1} = (Q-B) S_ij + (i S_{i-1,j} + j S_{i,j-1}) / (2 zeta),  S_00 = sqrt(pi/zeta) exp(-mu X^2)
// and -1/2 d^2/dx^2 acting on the ket: x^j e^{-b x^2} -> j(j-1) x^{j-2} - 2b(2j+1) x^j + 4b^2 x^{j+2}.
// ---------------------------------------------------------------------------------------------
template <int LA, int LB>
__global__ void __launch_bounds__(128) overlap_kinetic_kernel(ShellView bas, const int2* __restrict__ pairs,
                                                              int npairs, double* __restrict__ Sm,
                                                              double* __restrict__ Tm, int n) {
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npairs) return;
    const int2 pr = pairs[ip];
    const int a = pr.x, b = pr.y;
    double A[3], B[3];
    load3(bas.xyz, a, A);
    load3(bas.xyz, b, B);
    const double aa = bas.alpha[a], ab = bas.alpha[b];
    const double zeta = aa + ab, iz = 1.0 / zeta, mu = aa * ab * iz;
    constexpr int JM = LB + 2;
    double s[3][LA + 1][JM + 1];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double Q = (aa * A[d] + ab * B[d]) * iz;
        const double X = A[d] - B[d];
        const double qa = Q - A[d], qb = Q - B[d];
        s[d][0][0] = sqrt(PI * iz) * exp(-mu * X * X);
#pragma unroll
        for (int j = 0; j < JM; ++j)
            s[d][0][j + 1] = qb * s[d][0][j] + (j > 0 ? j * s[d][0][j - 1] : 0.0) * 0.5 * iz;
#pragma unroll
        for (int i = 0; i < LA; ++i)
#pragma unroll
            for (int j = 0; j <= JM; ++j)
                s[d][i + 1][j] = qa * s[d][i][j] +
                                 ((i > 0 ? i * s[d][i - 1][j] : 0.0) + (j > 0 ? j * s[d][i][j - 1] : 0.0)) * 0.5 * iz;
    }
    constexpr int CA = ncart(LA), CB = ncart(LB);
    double cs[CA * CB], ct[CA * CB];
#pragma unroll
    for (int i1 = LA; i1 >= 0; --i1)
#pragma unroll
        for (int j1 = LA - i1; j1 >= 0; --j1) {
            const int k1 = LA - i1 - j1;
            const int pa[3] = {i1, j1, k1};
#pragma unroll
            for (int i2 = LB; i2 >= 0; --i2)
#pragma unroll
                for (int j2 = LB - i2; j2 >= 0; --j2) {
                    const int k2 = LB - i2 - j2;
                    const int pb[3] = {i2, j2, k2};
                    double sd[3], td[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const int ia = pa[d], jb = pb[d];
                        sd[d] = s[d][ia][jb];
                        double d2 = 4.0 * ab * ab * s[d][ia][jb + 2] - 2.0 * ab * (2 * jb + 1) * s[d][ia][jb];
                        if (jb >= 2) d2 += jb * (jb - 1) * s[d][ia][jb - 2];
                        td[d] = -0.5 * d2;
                    }
                    const int idx = cidx(j1, k1) * CB + cidx(j2, k2);
                    cs[idx] = sd[0] * sd[1] * sd[2];
                    ct[idx] = td[0] * sd[1] * sd[2] + sd[0] * td[1] * sd[2] + sd[0] * sd[1] * td[2];
                }
        }
    double ss[nsph(LA) * nsph(LB)], st[nsph(LA) * nsph(LB)];
    cart_to_sph<0, LA, LB>(cs, ss);
    cart_to_sph<0, LA, LB>(ct, st);
    const double scale = bas.norm[a] * bas.norm[b];
    const int oa = bas.off[a], ob = bas.off[b];
#pragma unroll
    for (int i = 0; i < nsph(LA); ++i)
#pragma unroll
        for (int j = 0; j < nsph(LB); ++j) {
            const long long x = (long long)(oa + i) * n + ob + j, y = (long long)(ob + j) * n + oa + i;
            Sm[x] = Sm[y] = scale * ss[i * nsph(LB) + j];
            Tm[x] = Tm[y] = scale * st[i * nsph(LB) + j];
        }
}

inline int blocks_for(int count) { return (count + 127) / 128; }

}  // namespace

// ---------------------------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------------------------
void compute_one_electron(df_handle* h) {
    const double* tab = rys_table_device();
    ShellView bv = view(h->dbas);
    h->S.zero(h->stream);
    h->T.zero(h->stream);
    h->V.zero(h->stream);
    for (const ClassList& c : h->pair_classes) {
        if (c.count == 0) continue;
        dim3 grid(blocks_for(c.count));
#define OK_CASE(A, B)                                                                                          \
    if (c.la == A && c.lb == B) {                                                                              \
        overlap_kinetic_kernel<A, B><<<grid, 128, 0, h->stream>>>(bv, c.d_pairs, c.count, h->S.p, h->T.p, h->n); \
        nuclear_kernel<A, B><<<grid, 128, 0, h->stream>>>(bv, c.d_pairs, c.count, h->d_atom_xyz.p,              \
                                                          h->d_atom_Z.p, (int)h->atoms.size(), tab, h->V.p, h->n); \
    }
        OK_CASE(0, 0) OK_CASE(1, 0) OK_CASE(1, 1) OK_CASE(2, 0) OK_CASE(2, 1) OK_CASE(2, 2)
#undef OK_CASE
        DF_CHECK_LAUNCH();
    }
}

void compute_metric(df_handle* h) {
    const double* tab = rys_table_device();
    ShellView av = view(h->daux);
    h->metric.zero(h->stream);
    for (const ClassList& c : h->aux_pairs) {
        if (c.count == 0) continue;
        dim3 grid(blocks_for(c.count));
#define M_CASE(A, B) \
    if (c.la == A && c.lb == B) metric_kernel<A, B><<<grid, 128, 0, h->stream>>>(av, c.d_pairs, c.count, tab, h->metric.p, h->naux);
        M_CASE(0, 0) M_CASE(1, 0) M_CASE(1, 1) M_CASE(2, 0) M_CASE(2, 1) M_CASE(2, 2)
        M_CASE(3, 0) M_CASE(3, 1) M_CASE(3, 2) M_CASE(3, 3)
#undef M_CASE
        DF_CHECK_LAUNCH();
    }
}

void compute_three_center(df_handle* h, double* out, double tau) {
    (void)tau;
    const double* tab = rys_table_device();
    ShellView bv = view(h->dbas), av = view(h->daux);
    DF_CUDA(cudaMemsetAsync(out, 0, (size_t)h->naux * h->pk.row * sizeof(double), h->stream));
    for (int lp = 0; lp <= DF_LMAX_AUX; ++lp) {
        const int na = (int)h->aux_by_l[lp].size();
        if (na == 0) continue;
        const int* auxl = h->d_aux_by_l[lp].p;
        for (const ClassList& c : h->pair_classes) {
            if (c.count == 0) continue;
            dim3 grid(blocks_for(c.count), na < 65535 ? na : 65535);
#define E_CASE(P, A, B)                                                                                    \
    if (lp == P && c.la == A && c.lb == B)                                                                 \
        eri3c_kernel<P, A, B><<<grid, 128, 0, h->stream>>>(bv, av, c.d_pairs, c.count, auxl, na, tab, out, \
                                                           h->pk.row);
#define E_ROW(P) E_CASE(P, 0, 0) E_CASE(P, 1, 0) E_CASE(P, 1, 1) E_CASE(P, 2, 0) E_CASE(P, 2, 1) E_CASE(P, 2, 2)
            E_ROW(0) E_ROW(1) E_ROW(2) E_ROW(3)
#undef E_ROW
#undef E_CASE
            DF_CHECK_LAUNCH();
        }
    }
}

}  // namespace dfhf
