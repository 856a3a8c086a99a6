// Integral kernels: three-centre (P|mu nu) (the integral hot loop), the two-centre Coulomb metric
// (P|Q), and the one-electron overlap, kinetic and nuclear-attraction matrices.
//
// Paper, section "Molecular integrals": the 1/r12 integrals are computed by Rys quadrature over shell
// objects, and the nuclear attraction needs the molecule as well. One kernel is instantiated per
// angular-momentum class; one thread evaluates one shell triple (or shell pair) with rys_eri.cuh.
#include <algorithm>
#include <cmath>
#include <vector>

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
// three-centre (P|ab) of one shell triple: pair (a, b) of class (LA, LB), auxiliary shell P of
// angular momentum LP; written into rows of `row` doubles, packed mu >= nu tiles
// ---------------------------------------------------------------------------------------------
template <int LP, int LA, int LB>
__device__ __forceinline__ void eri3c_triple(const ShellView& bas, const ShellView& aux, int a, int b, const double* A,
                                             const double* B, int P, const double* __restrict__ tab,
                                             double* __restrict__ out, long long row) {
    const double aa = bas.alpha[a], ab = bas.alpha[b];
    const double nab = bas.norm[a] * bas.norm[b];
    const int offa = bas.off[a], offb = bas.off[b];
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

// threads over orbital shell pairs of one class, blockIdx.y over auxiliary shells of angular momentum LP
template <int LP, int LA, int LB>
__global__ void __launch_bounds__(128) eri3c_kernel(ShellView bas, ShellView aux, const int2* __restrict__ pairs,
                                                    int npairs, const int* __restrict__ auxl, int naux_l,
                                                    const double* __restrict__ tab, double* __restrict__ out,
                                                    long long row) {
    const int ip = blockIdx.x * blockDim.x + threadIdx.x;
    if (ip >= npairs) return;
    const int2 pr = pairs[ip];
    double A[3], B[3];
    load3(bas.xyz, pr.x, A);
    load3(bas.xyz, pr.y, B);
    for (int ia = blockIdx.y; ia < naux_l; ia += gridDim.y)
        eri3c_triple<LP, LA, LB>(bas, aux, pr.x, pr.y, A, B, auxl[ia], tab, out, row);
}

// ---------------------------------------------------------------------------------------------
// three-centre integrals of many molecules in one persistent launch per class: a global queue of work
// items (molecule, block of 128 shell pairs, block of AUX_PER_ITEM auxiliary shells), taken in order by
// resident CTAs through an atomic counter; the molecule of an item is found by binary search over the
// prefix sums of the molecules' item counts.
// ---------------------------------------------------------------------------------------------
constexpr int AUX_PER_ITEM = 8;

struct Mol3c {
    ShellView bas, aux;
    const int2* pairs;       // the class's pair list
    int npairs;
    const int* auxl;         // auxiliary shells of angular momentum LP
    int naux_l;
    double* out;
    long long row;
};

template <int LP, int LA, int LB>
__global__ void __launch_bounds__(128) eri3c_grouped_kernel(const Mol3c* __restrict__ mols,
                                                            const long long* __restrict__ item_off, int nmol,
                                                            unsigned long long* __restrict__ counter,
                                                            const double* __restrict__ tab) {
    __shared__ long long s_item;
    const long long total = item_off[nmol];
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long item = s_item;
        __syncthreads();
        if (item >= total) return;
        int lo = 0, hi = nmol;   // the molecule m with item_off[m] <= item < item_off[m + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) / 2;
            if (item_off[mid] <= item) lo = mid;
            else hi = mid;
        }
        const Mol3c& M = mols[lo];
        const long long local = item - item_off[lo];
        const int npb = (M.npairs + 127) / 128;
        const int pb = (int)(local % npb), ab = (int)(local / npb);
        const int ip = pb * 128 + threadIdx.x;
        if (ip < M.npairs) {
            const int2 pr = M.pairs[ip];
            double A[3], B[3];
            load3(M.bas.xyz, pr.x, A);
            load3(M.bas.xyz, pr.y, B);
            const int a1 = min(M.naux_l, (ab + 1) * AUX_PER_ITEM);
            for (int ia = ab * AUX_PER_ITEM; ia < a1; ++ia)
                eri3c_triple<LP, LA, LB>(M.bas, M.aux, pr.x, pr.y, A, B, M.auxl[ia], tab, M.out, M.row);
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

// Three-centre integrals of several molecules (outs[i]: rows of hs[i]->pk.row doubles, zeroed here) on
// stream s: one persistent launch per angular-momentum class over all molecules' work items. The work
// descriptors of every class are staged once; the call returns when the work is enqueued.
void compute_three_center_grouped(const std::vector<df_handle*>& hs, const std::vector<double*>& outs,
                                  cudaStream_t s) {
    const int nmol = (int)hs.size();
    if (nmol == 0) return;
    const double* tab = rys_table_device();
    int dev = 0, sms = 0;
    DF_CUDA(cudaGetDevice(&dev));
    DF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (int i = 0; i < nmol; ++i)
        DF_CUDA(cudaMemsetAsync(outs[i], 0, (size_t)hs[i]->naux * hs[i]->pk.row * sizeof(double), s));
    constexpr int NCLS = (DF_LMAX_AUX + 1) * 6;   // (lP, la >= lb) classes
    std::vector<Mol3c> mols((size_t)NCLS * nmol);
    std::vector<long long> off((size_t)NCLS * (nmol + 1));
    for (int lp = 0; lp <= DF_LMAX_AUX; ++lp)
        for (int ci = 0; ci < 6; ++ci) {                  // pair_classes order: la ascending, lb <= la
            const int k = lp * 6 + ci;
            long long* o = &off[(size_t)k * (nmol + 1)];
            o[0] = 0;
            for (int i = 0; i < nmol; ++i) {
                df_handle* h = hs[i];
                const ClassList& c = h->pair_classes[ci];
                const int na = (int)h->aux_by_l[lp].size();
                mols[(size_t)k * nmol + i] = Mol3c{view(h->dbas), view(h->daux), c.d_pairs, c.count,
                                                   h->d_aux_by_l[lp].p, na, outs[i], h->pk.row};
                const long long items =
                    (c.count > 0 && na > 0) ? (long long)((c.count + 127) / 128) * ((na + AUX_PER_ITEM - 1) / AUX_PER_ITEM)
                                            : 0;
                o[i + 1] = o[i] + items;
            }
        }
    DevBuf<Mol3c> dmols;
    DevBuf<long long> doff;
    DevBuf<unsigned long long> dcounter;
    dmols.alloc(mols.size());
    doff.alloc(off.size());
    dcounter.alloc(NCLS);
    DF_CUDA(cudaMemcpyAsync(dmols.p, mols.data(), sizeof(Mol3c) * mols.size(), cudaMemcpyHostToDevice, s));
    DF_CUDA(cudaMemcpyAsync(doff.p, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, s));
    DF_CUDA(cudaMemsetAsync(dcounter.p, 0, sizeof(unsigned long long) * NCLS, s));
    for (int lp = 0; lp <= DF_LMAX_AUX; ++lp)
        for (int la = 0; la <= DF_LMAX_ORB; ++la)
            for (int lb = 0; lb <= la; ++lb) {
                const int k = lp * 6 + la * (la + 1) / 2 + lb;
                const long long total = off[(size_t)k * (nmol + 1) + nmol];
                if (total == 0) continue;
                const unsigned grid = (unsigned)std::min<long long>(total, (long long)sms * 8);
                const Mol3c* dm = dmols.p + (size_t)k * nmol;
                const long long* doffk = doff.p + (size_t)k * (nmol + 1);
#define G_CASE(P, A, B)                                                                                   \
    if (lp == P && la == A && lb == B)                                                                    \
        eri3c_grouped_kernel<P, A, B><<<grid, 128, 0, s>>>(dm, doffk, nmol, dcounter.p + k, tab);
#define G_ROW(P) G_CASE(P, 0, 0) G_CASE(P, 1, 0) G_CASE(P, 1, 1) G_CASE(P, 2, 0) G_CASE(P, 2, 1) G_CASE(P, 2, 2)
                G_ROW(0) G_ROW(1) G_ROW(2) G_ROW(3)
#undef G_ROW
#undef G_CASE
                DF_CHECK_LAUNCH();
            }
    DF_CUDA(cudaStreamSynchronize(s));   // the staging buffers are released on return
}

}  // namespace dfhf
