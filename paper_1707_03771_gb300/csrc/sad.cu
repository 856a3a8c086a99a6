// Superposition-of-atomic-densities (SAD) initial guess. The paper names no initial guess; the reading:
//   * each element gets a spherically averaged, fractional-occupation restricted DF-HF of the neutral
//     atom in the atom's own orbital and auxiliary shells (the shells the molecule assigns to it): Aufbau
//     occupations in which a set of degenerate orbitals shares its electrons equally, F = H + J[D] - K with
//     K the orbital-form exchange of the orbitals weighted by sqrt(n_i / 2) (half the exchange of D);
//   * the molecule's guess density is the block-diagonal assembly of its atoms' densities, scaled so that
//     tr(D S) = N electrons.
// The guess is carried as a factor C0 (n x m, m = total occupied atomic orbitals) with D0 = 2 C0 C0^T, so
// that the first Fock matrix, exchange included, is built from D0 itself (eqs. 1-3 need the factor).
// Each atomic SCF runs on the GPU through the library's own handle, integrals, J/K and SCF driver; their
// factors are kept for the process per atom signature (element and shells relative to the nucleus).
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>

#include "common.cuh"

namespace dfhf {

namespace {

struct AtomFactor {
    int n = 0, m = 0;
    std::vector<double> Cw;   // n x m, row-major
};

std::mutex g_sad_mu;
std::map<std::string, AtomFactor> g_sad_cache;

std::string signature(const df_atom& at, const std::vector<df_shell>& basis, const std::vector<df_shell>& aux) {
    std::string key = "Z" + std::to_string(at.Z);
    char buf[160];
    for (const auto* list : {&basis, &aux}) {
        key += "|";
        for (const df_shell& sh : *list) {
            std::snprintf(buf, sizeof buf, "%d:%.17g:%.17g:%.17g:%.17g;", sh.l, sh.exponent, sh.center[0] - at.xyz[0],
                          sh.center[1] - at.xyz[1], sh.center[2] - at.xyz[2]);
            key += buf;
        }
    }
    return key;
}

// sum_i a[i] b[i] (single block, deterministic)
__global__ void dot_kernel(const double* __restrict__ a, const double* __restrict__ b, long long len,
                           double* __restrict__ out) {
    double s = 0.0;
    for (long long i = threadIdx.x; i < len; i += blockDim.x) s = fma(a[i], b[i], s);
    __shared__ double sm[256];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

__global__ void scale_kernel(double* __restrict__ x, long long len, const double* __restrict__ dot, double nelec) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) x[i] *= sqrt(nelec / (2.0 * *dot));   // tr(D0 S) = 2 tr(C0^T S C0)
}

}  // namespace

void sad_factor(df_handle* h, DevBuf<double>& C0, int& m0) {
    const int natom = (int)h->atoms.size();
    std::vector<int> shell_off(h->basis.size() + 1, 0);
    for (size_t i = 0; i < h->basis.size(); ++i) shell_off[i + 1] = shell_off[i] + 2 * h->basis[i].l + 1;
    struct Block {
        std::vector<int> rows;   // molecule function of each atomic function
        const AtomFactor* f;
    };
    std::vector<Block> blocks;
    m0 = 0;
    for (int a = 0; a < natom; ++a) {
        const df_atom& at = h->atoms[a];
        std::vector<df_shell> basis, aux;
        std::vector<int> rows;
        for (size_t i = 0; i < h->basis.size(); ++i)
            if (h->basis[i].atom == a) {
                df_shell sh = h->basis[i];
                sh.atom = 0;
                basis.push_back(sh);
                for (int f = shell_off[i]; f < shell_off[i + 1]; ++f) rows.push_back(f);
            }
        for (const df_shell& sa : h->aux)
            if (sa.atom == a) {
                df_shell sh = sa;
                sh.atom = 0;
                aux.push_back(sh);
            }
        if (at.Z <= 0 || basis.empty()) continue;   // ghost atoms and atoms without functions: no block
        if (aux.empty())
            throw Error{DF_E_ARG, "superposition-of-atomic-densities guess: atom " + std::to_string(a) +
                                      " has orbital shells but no auxiliary shells (shells are matched to atoms by "
                                      "their atom field)"};
        const std::string key = signature(at, basis, aux);
        const AtomFactor* fac = nullptr;
        {
            std::lock_guard<std::mutex> lock(g_sad_mu);
            auto it = g_sad_cache.find(key);
            if (it != g_sad_cache.end()) fac = &it->second;
        }
        if (!fac) {
            df_handle* ha = nullptr;
            const int rc = init_handle(&at, 1, basis.data(), (int)basis.size(), aux.data(), (int)aux.size(), 0, &ha,
                                       false);
            if (rc != DF_OK)
                throw Error{rc, "superposition-of-atomic-densities guess: handle for atom " + std::to_string(a)};
            AtomFactor af;
            af.n = ha->n;
            try {
                atomic_scf(ha, (double)at.Z, af.Cw, af.m);
            } catch (...) {
                df_free(ha);
                throw;
            }
            df_free(ha);
            DF_CUDA(cudaSetDevice(h->device));
            std::lock_guard<std::mutex> lock(g_sad_mu);
            fac = &g_sad_cache.emplace(key, std::move(af)).first->second;   // map nodes do not move
        }
        blocks.push_back(Block{rows, fac});
        m0 += fac->m;
    }
    if (m0 == 0) throw Error{DF_E_ARG, "superposition-of-atomic-densities guess: no atom carries functions"};
    const int n = h->n;
    std::vector<double> host((size_t)n * m0, 0.0);
    int col = 0;
    for (const Block& b : blocks) {
        for (size_t r = 0; r < b.rows.size(); ++r)
            for (int j = 0; j < b.f->m; ++j) host[(size_t)b.rows[r] * m0 + col + j] = b.f->Cw[r * b.f->m + j];
        col += b.f->m;
    }
    cudaStream_t s = h->stream;
    C0.alloc(host.size());
    DevBuf<double> T, dot;
    T.alloc(host.size());
    dot.alloc(1);
    DF_CUDA(cudaMemcpyAsync(C0.p, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice, s));
    // scaled to tr(D0 S) = N: 2 sum C0 .* (S C0) is tr(D0 S)
    dgemm(s, false, false, n, m0, n, 1.0, h->S.p, n, C0.p, m0, 0.0, T.p, m0);
    dot_kernel<<<1, 256, 0, s>>>(C0.p, T.p, (long long)host.size(), dot.p);
    DF_CHECK_LAUNCH();
    scale_kernel<<<(unsigned)((host.size() + 255) / 256), 256, 0, s>>>(C0.p, (long long)host.size(), dot.p,
                                                                       (double)h->nelec);
    DF_CHECK_LAUNCH();
    DF_CUDA(cudaStreamSynchronize(s));   // host staging and T are released on return
}

}  // namespace dfhf

using namespace dfhf;

extern "C" int df_sad_density(df_handle* h, double* D0) {
    if (!h || !D0) return DF_E_ARG;
    try {
        DF_CUDA(cudaSetDevice(h->device));
        DevBuf<double> C0, D;
        int m0 = 0;
        sad_factor(h, C0, m0);
        D.alloc((size_t)h->n * h->n);
        dgemm(h->stream, false, true, h->n, h->n, m0, 2.0, C0.p, m0, C0.p, m0, 0.0, D.p, h->n);
        DF_CUDA(cudaMemcpyAsync(D0, D.p, sizeof(double) * h->n * h->n, cudaMemcpyDeviceToHost, h->stream));
        DF_CUDA(cudaStreamSynchronize(h->stream));
    } catch (const Error& e) {
        h->last_error = e.msg;
        return e.code;
    }
    return DF_OK;
}
