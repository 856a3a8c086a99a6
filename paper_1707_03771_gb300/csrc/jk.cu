// Per-iteration Coulomb and exchange builds from the packed, whitened B (paper eqs. 1-3).
//
// J (eq. 3): gamma_P = sum_{mu nu} B_{P,mu nu} D_{mu nu} is a dot product of each packed row of B
// with the packed, weighted density Dw (off-diagonal tiles carry weight 2, diagonal tiles are stored
// in full with weight 1), reduced with warp shuffles; J_{mu nu} = sum_P gamma_P B_{P,mu nu} is a
// column sweep over B with coalesced 16-byte loads. Both read B once; on GB300 both are bounded by
// the FP64 pipe (one FMA per 8 bytes needs 0.85 TFMA/s at 6.8 TB/s, above the ~0.5 TFMA/s DFMA rate).
// K (eqs. 1-2, first forms): Y = B C_occ per auxiliary row (dense.cu), then K = sum_P Y_P Y_P^T.
#include <algorithm>

#include "common.cuh"

namespace dfhf {

void y_transform_fp64(cudaStream_t s, const double* B, long long row, int nt, int naux, const double* Cp, int ldy,
                      int ncol, double* Y);
void k_syrk_fp64(cudaStream_t s, const double* Y, int naux, int np, int ldy, int ncol, int nsplit,
                 const int2* tiles, int ntiles, double* Kpart, int n, double* K);

namespace {

// Dw[packed(mu, nu)] = w D[mu][nu]; one block per tile pair (blockIdx.x = I, blockIdx.y = J)
__global__ void pack_density_kernel(const double* __restrict__ D, int n, double* __restrict__ Dw) {
    const int I = blockIdx.x, J = blockIdx.y;
    if (J > I) return;
    const double wgt = (I == J) ? 1.0 : 2.0;
    double* t = Dw + tile_pair(I, J) * TS * TS;
    for (int e = threadIdx.x; e < TS * TS; e += blockDim.x) {
        const int mu = I * TS + e / TS, nu = J * TS + e % TS;
        t[e] = (mu < n && nu < n) ? wgt * D[(long long)mu * n + nu] : 0.0;
    }
}

// M[mu][nu] (n x n) from a packed row
__global__ void unpack_kernel(const double* __restrict__ packed, int n, double* __restrict__ M) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    M[idx] = packed[packed_index((int)(idx / n), (int)(idx % n))];
}

// gamma_P = <B_P, Dw>: one block per row, 16-byte loads, shuffle + shared reduction
__global__ void __launch_bounds__(256) gamma_kernel(const double* __restrict__ B, long long row,
                                                    const double* __restrict__ Dw, double* __restrict__ gamma) {
    const long long P = blockIdx.x;
    const double2* b = reinterpret_cast<const double2*>(B + P * row);
    const double2* d = reinterpret_cast<const double2*>(Dw);
    const long long n2 = row / 2;
    double s0 = 0.0, s1 = 0.0;
    for (long long i = threadIdx.x; i < n2; i += blockDim.x) {
        const double2 x = __ldcs(b + i);
        const double2 y = __ldg(d + i);
        s0 = fma(x.x, y.x, s0);
        s1 = fma(x.y, y.y, s1);
    }
    double s = s0 + s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? part[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) gamma[P] = s;
    }
}

// Jp[x] = sum_P gamma_P B[P][x]; each thread owns two adjacent columns, blockIdx.y splits P
__global__ void __launch_bounds__(256) coulomb_kernel(const double* __restrict__ B, long long row, int naux,
                                                      const double* __restrict__ gamma, int nsplit,
                                                      double* __restrict__ Jpart) {
    const long long c2 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c2 * 2 >= row) return;
    const int s = blockIdx.y;
    const int p0 = (int)((long long)naux * s / nsplit), p1 = (int)((long long)naux * (s + 1) / nsplit);
    double a0 = 0.0, a1 = 0.0;
    for (int P = p0; P < p1; ++P) {
        const double2 x = __ldcs(reinterpret_cast<const double2*>(B + (long long)P * row) + c2);
        const double g = gamma[P];
        a0 = fma(g, x.x, a0);
        a1 = fma(g, x.y, a1);
    }
    reinterpret_cast<double2*>(Jpart + (long long)s * row)[c2] = make_double2(a0, a1);
}

__global__ void sum_splits_kernel(const double* __restrict__ part, int nsplit, long long len, double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    double s = 0.0;
    for (int t = 0; t < nsplit; ++t) s += part[(long long)t * len + i];
    out[i] = s;
}

// Cpad[mu][i] = C[mu][i] for mu < n, i < nocc; zero elsewhere (np x ldy)
__global__ void pad_c_kernel(const double* __restrict__ C, int n, int nocc, int np, int ldy, double* __restrict__ Cp) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)np * ldy) return;
    const int mu = (int)(idx / ldy), i = (int)(idx % ldy);
    Cp[idx] = (mu < n && i < nocc) ? C[(long long)mu * nocc + i] : 0.0;
}

constexpr int J_SPLIT = 8;

}  // namespace

int k_splits(const df_handle* h) {
    const int tiles = h->pk.nt * (h->pk.nt + 1) / 2;
    int s = (4 * 152 + tiles - 1) / tiles;
    return std::max(1, std::min(s, std::max(1, h->naux / 4)));
}

void ensure_jk_buffers(df_handle* h, int nocc) {
    const Packing& pk = h->pk;
    if (!h->Dw.p) {
        h->Dw.alloc(pk.row);
        h->gamma.alloc(h->naux);
        h->Jp.alloc(pk.row * (J_SPLIT + 1));
        h->dD.alloc((size_t)h->n * h->n);
        h->dJ.alloc((size_t)h->n * h->n);
        h->dK.alloc((size_t)h->n * h->n);
        h->Kpart.alloc((size_t)k_splits(h) * pk.np * pk.np);
        // tile list for the exchange contraction: lower tile pairs
        std::vector<int2> tiles;
        for (int I = 0; I < pk.nt; ++I)
            for (int J = 0; J <= I; ++J) tiles.push_back(make_int2(I, J));
        h->ktiles.alloc(tiles.size());
        DF_CUDA(cudaMemcpyAsync(h->ktiles.p, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, h->stream));
    }
    if (nocc > h->nocc_alloc) {
        const int ldy = ((nocc + 31) / 32) * 32;
        h->Cpad.alloc((size_t)pk.np * ldy);
        h->dC.alloc((size_t)h->n * nocc);
        h->nocc_alloc = nocc;
    }
}

void coulomb_fp64(df_handle* h, const double* dD, double* dJ) {
    const Packing& pk = h->pk;
    cudaStream_t s = h->stream;
    PhaseTimer t(h->sync_timing, 3);
    pack_density_kernel<<<dim3(pk.nt, pk.nt), 256, 0, s>>>(dD, h->n, h->Dw.p);
    DF_CHECK_LAUNCH();
    t.mark(0, s);
    gamma_kernel<<<h->naux, 256, 0, s>>>(h->B.p, pk.row, h->Dw.p, h->gamma.p);
    DF_CHECK_LAUNCH();
    t.mark(1, s);
    const long long c2 = pk.row / 2;
    coulomb_kernel<<<dim3((unsigned)((c2 + 255) / 256), J_SPLIT), 256, 0, s>>>(h->B.p, pk.row, h->naux, h->gamma.p,
                                                                             J_SPLIT, h->Jp.p + pk.row);
    DF_CHECK_LAUNCH();
    t.mark(2, s);
    sum_splits_kernel<<<(unsigned)((pk.row + 255) / 256), 256, 0, s>>>(h->Jp.p + pk.row, J_SPLIT, pk.row, h->Jp.p);
    DF_CHECK_LAUNCH();
    const long long nn = (long long)h->n * h->n;
    unpack_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(h->Jp.p, h->n, dJ);
    DF_CHECK_LAUNCH();
    if (t.on) {
        t.sync(2);
        h->timings_ms[4] = t.ms(0, 1);
        h->timings_ms[5] = t.ms(1, 2);
    }
}

void pad_occupied(df_handle* h, const double* dC, int nocc, int ldy) {
    const long long tot = (long long)h->pk.np * ldy;
    pad_c_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(dC, h->n, nocc, h->pk.np, ldy, h->Cpad.p);
    DF_CHECK_LAUNCH();
}

void exchange_fp64(df_handle* h, int nocc, double* dK) {
    const Packing& pk = h->pk;
    cudaStream_t s = h->stream;
    const int ldy = ((nocc + 31) / 32) * 32;
    PhaseTimer t(h->sync_timing, 3);
    t.mark(0, s);
    h->exchange_launches = 3;   // Y transform, K contraction, K reduction
    // Y (naux x np x ldy doubles): the split exchange's Y buffer when the handle has one large enough (8 bytes
    // per element as well; both run in order on the handle's stream), else its own, allocated on first use
    const size_t ny = (size_t)h->naux * pk.np * ldy;
    double* Y = split_y_buffer(h, (long long)ny);
    if (!Y) {
        if (h->Y.n < ny) h->Y.alloc(ny);
        Y = h->Y.p;
    }
    y_transform_fp64(s, h->B.p, pk.row, pk.nt, h->naux, h->Cpad.p, ldy, nocc, Y);
    t.mark(1, s);
    const int ntiles = pk.nt * (pk.nt + 1) / 2;
    k_syrk_fp64(s, Y, h->naux, pk.np, ldy, nocc, k_splits(h), h->ktiles.p, ntiles, h->Kpart.p, h->n, dK);
    t.mark(2, s);
    if (t.on) {
        t.sync(2);
        h->timings_ms[6] = t.ms(0, 1);
        h->timings_ms[7] = t.ms(1, 2);
    }
}

void jk_fp64(df_handle* h, const double* dD, const double* dC, int nocc, double* dJ, double* dK) {
    ensure_jk_buffers(h, nocc);
    coulomb_fp64(h, dD, dJ);
    pad_occupied(h, dC, nocc, ((nocc + 31) / 32) * 32);
    exchange_fp64(h, nocc, dK);
}

void unpack_rows(df_handle* h, const double* packed, int p0, int count, double* dout) {
    const long long nn = (long long)h->n * h->n;
    for (int r = 0; r < count; ++r) {
        unpack_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, h->stream>>>(packed + (long long)(p0 + r) * h->pk.row,
                                                                          h->n, dout + r * nn);
        DF_CHECK_LAUNCH();
    }
}

double elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    DF_CUDA(cudaEventElapsedTime(&ms, a, b));
    return ms;
}

}  // namespace dfhf

namespace dfhf {

// The Coulomb build with every scratch buffer supplied by the caller and no split of the auxiliary
// sum: Dw and Jp hold `row` doubles each, gamma `naux`. Each scratch element is written before it
// is read within the call, so nothing has to start at zero. No allocation, no synchronisation.
// Loads the Coulomb kernels on the current device now (under lazy module loading they would otherwise be
// loaded, and their code placed in device memory, at their first launch)
void coulomb_kernels_load() {
    cudaFuncAttributes a;
    DF_CUDA(cudaFuncGetAttributes(&a, pack_density_kernel));
    DF_CUDA(cudaFuncGetAttributes(&a, gamma_kernel));
    DF_CUDA(cudaFuncGetAttributes(&a, coulomb_kernel));
    DF_CUDA(cudaFuncGetAttributes(&a, unpack_kernel));
}

void coulomb_with_scratch(cudaStream_t s, const double* B, const Packing& pk, int naux, int n, const double* dD,
                          double* dJ, double* Dw, double* gamma, double* Jp) {
    pack_density_kernel<<<dim3(pk.nt, pk.nt), 256, 0, s>>>(dD, n, Dw);
    DF_CHECK_LAUNCH();
    gamma_kernel<<<naux, 256, 0, s>>>(B, pk.row, Dw, gamma);
    DF_CHECK_LAUNCH();
    const long long c2 = pk.row / 2;
    coulomb_kernel<<<dim3((unsigned)((c2 + 255) / 256), 1), 256, 0, s>>>(B, pk.row, naux, gamma, 1, Jp);
    DF_CHECK_LAUNCH();
    const long long nn = (long long)n * n;
    unpack_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(Jp, n, dJ);
    DF_CHECK_LAUNCH();
}

}  // namespace dfhf
