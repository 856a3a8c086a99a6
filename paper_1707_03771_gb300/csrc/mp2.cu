// Density-fitted closed-shell MP2 correlation energy (the paper lists MP2 among the programs on the
// density-fitting utilities, section "Program features"), FP64 on the GPU from the handle's B:
//   * Y_{P,mu i} = sum_nu B_{P,mu nu} C_{nu i} (eq. 1, first form; the FP64 half-transform of the exchange);
//   * B^P_{ia} = sum_mu C_{mu a} Y_{P,mu i} (eq. 1 again, on the second index), stored as T[i][a][P];
//   * for each occupied i, V_{ia,jb} = sum_P B^P_{ia} B^P_{jb} for every j <= i in one product
//     (eq. 2, second form);
//   * E2 = sum_{ij ab} (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b), every orbital correlated,
//     each pair's sum in one block (fixed order) and the pairs added on the host in a fixed order.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace dfhf {

namespace {

inline unsigned nb256(long long n) { return (unsigned)((n + 255) / 256); }

// Bia[P][a][i] (P < naux, a < nvir, i < nocc) -> T[i][a][P]
__global__ void ov_transpose_kernel(const double* __restrict__ Bia, int naux, int nvir, int nocc,
                                    double* __restrict__ T) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)naux * nvir * nocc;
    if (idx >= total) return;
    const int P = (int)(idx % naux);
    const long long r = idx / naux;
    const int a = (int)(r % nvir);
    const int i = (int)(r / nvir);
    T[idx] = Bia[((long long)P * nvir + a) * nocc + i];
}

// pair energies of occupied i with every j <= i: V holds (ia|jb) at V[a][j nvir + b] (row stride ld);
// pe[j] = f sum_ab V_ab (2 V_ab - V_ba) / (e_i + e_j - e_a - e_b), f = 2 for j < i (the pair (j, i) too)
__global__ void __launch_bounds__(256) pair_energy_kernel(const double* __restrict__ V, long long ld, int i, int nocc,
                                                          int nvir, const double* __restrict__ eps,
                                                          double* __restrict__ pe) {
    const int j = blockIdx.x;
    const double eij = eps[i] + eps[j];
    const double* ev = eps + nocc;
    double s = 0.0;
    for (long long ab = threadIdx.x; ab < (long long)nvir * nvir; ab += blockDim.x) {
        const int a = (int)(ab / nvir), b = (int)(ab % nvir);
        const double vab = V[(long long)a * ld + (long long)j * nvir + b];
        const double vba = V[(long long)b * ld + (long long)j * nvir + a];
        s += vab * (2.0 * vab - vba) / (eij - ev[a] - ev[b]);
    }
    __shared__ double sm[256];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) pe[j] = (j < i ? 2.0 : 1.0) * sm[0];
}

}  // namespace

double mp2_energy(df_handle* h, const double* C_host, const double* eps_host, int nmo, int nocc) {
    const int n = h->n, naux = h->naux, nvir = nmo - nocc;
    const Packing& pk = h->pk;
    cudaStream_t s = h->stream;
    const int ldy = ((nocc + 31) / 32) * 32;
    ensure_jk_buffers(h, nocc);
    DevBuf<double> Call, Cocc, Cvir, eps, Y, Bia, T, V, pe;
    Call.alloc((size_t)n * nmo);
    Cocc.alloc((size_t)n * nocc);
    Cvir.alloc((size_t)n * nvir);
    eps.alloc(nmo);
    DF_CUDA(cudaMemcpyAsync(Call.p, C_host, sizeof(double) * n * nmo, cudaMemcpyHostToDevice, s));
    DF_CUDA(cudaMemcpyAsync(eps.p, eps_host, sizeof(double) * nmo, cudaMemcpyHostToDevice, s));
    DF_CUDA(cudaMemcpy2DAsync(Cocc.p, sizeof(double) * nocc, Call.p, sizeof(double) * nmo, sizeof(double) * nocc, n,
                              cudaMemcpyDeviceToDevice, s));
    DF_CUDA(cudaMemcpy2DAsync(Cvir.p, sizeof(double) * nvir, Call.p + nocc, sizeof(double) * nmo, sizeof(double) * nvir,
                              n, cudaMemcpyDeviceToDevice, s));
    // Y = B C_occ over the padded orbital rows (rows beyond n are zero)
    pad_occupied(h, Cocc.p, nocc, ldy);
    Y.alloc((size_t)naux * pk.np * ldy);
    y_transform_fp64(s, h->B.p, pk.row, pk.nt, naux, h->Cpad.p, ldy, nocc, Y.p);
    // B^P_ia = C_vir^T Y_P for every P, then T[i][a][P]
    Bia.alloc((size_t)naux * nvir * nocc);
    for (int P = 0; P < naux; ++P)
        dgemm(s, true, false, nvir, nocc, n, 1.0, Cvir.p, nvir, Y.p + (long long)P * pk.np * ldy, ldy, 0.0,
              Bia.p + (long long)P * nvir * nocc, nocc);
    Y.release();
    T.alloc((size_t)naux * nvir * nocc);
    ov_transpose_kernel<<<nb256((long long)naux * nvir * nocc), 256, 0, s>>>(Bia.p, naux, nvir, nocc, T.p);
    DF_CHECK_LAUNCH();
    Bia.release();
    // rows of pair integrals: V = T_i T_{0..i}^T (nvir x (i + 1) nvir) and the pair energies of row i
    V.alloc((size_t)nvir * nocc * nvir);
    pe.alloc((size_t)nocc * nocc);
    pe.zero(s);
    for (int i = 0; i < nocc; ++i) {
        const long long ld = (long long)(i + 1) * nvir;
        dgemm(s, false, true, nvir, (int)ld, naux, 1.0, T.p + (long long)i * nvir * naux, naux, T.p, naux, 0.0, V.p,
              (int)ld);
        pair_energy_kernel<<<i + 1, 256, 0, s>>>(V.p, ld, i, nocc, nvir, eps.p, pe.p + (long long)i * nocc);
        DF_CHECK_LAUNCH();
    }
    std::vector<double> host((size_t)nocc * nocc);
    DF_CUDA(cudaMemcpyAsync(host.data(), pe.p, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, s));
    DF_CUDA(cudaStreamSynchronize(s));
    double e2 = 0.0;
    for (int i = 0; i < nocc; ++i)
        for (int j = 0; j <= i; ++j) e2 += host[(size_t)i * nocc + j];
    return e2;
}

}  // namespace dfhf

using namespace dfhf;

extern "C" int df_mp2(df_handle* h, const double* C, const double* eps, int nmo, int nocc, double* e2) {
    if (!h || !C || !eps || !e2 || nocc < 1 || nmo <= nocc || nmo > h->n) return DF_E_ARG;
    if (!h->built || !h->B.p) {
        h->last_error = "df_mp2: B not built";
        return DF_E_STATE;
    }
    try {
        DF_CUDA(cudaSetDevice(h->device));
        *e2 = mp2_energy(h, C, eps, nmo, nocc);
    } catch (const Error& e) {
        h->last_error = e.msg;
        return e.code;
    }
    return DF_OK;
}
