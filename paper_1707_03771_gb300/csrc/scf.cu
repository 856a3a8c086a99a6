// Restricted Hartree-Fock driver on the GPU (paper, section "Standard algorithms": RHF built on the
// density-fitted Fock builder). The paper gives no SCF details; this follows the textbook scheme:
//   canonical orthogonalisation X = U s^{-1/2} (eigenvalues of S below 1e-7 dropped),
//   core-Hamiltonian guess, F = H + J - K, E = tr(DH) + 1/2 tr(DJ) - 1/2 tr(DK) + E_nuc,
//   Pulay DIIS on e = X^T (F D S - S D F) X, Roothaan step X^T F X = V eps V^T, C = X V,
//   D = 2 C_occ C_occ^T (Aufbau), converged when |dE| < conv_E and max|e| < conv_err.
// Every step runs on the device in FP64 (DIIS included); only the energy and max|e| cross to the
// host each iteration for the convergence test. The symmetric eigensolver is cuSOLVER's dsyevd.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace dfhf {

void jk_dispatch(df_handle* h, const double* dD, const double* dC, int nocc, double* dJ, double* dK, int precision,
                 int slices);
void build_B(df_handle* h, double tau, bool keep);

namespace {

constexpr int DIIS_MAX = 16;
constexpr int SPLIT_LATE_SLICES = 5;      // slices of the late split-precision exchange builds
constexpr double SPLIT_RAMP_ERR = 1e-4;   // max|e| below which the late builds start

__global__ void build_x_kernel(const double* __restrict__ U, const double* __restrict__ s, int n, int first, int nX,
                               double* __restrict__ X) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * nX) return;
    const int mu = (int)(idx / nX), k = (int)(idx % nX);
    // U is the row-major view of cuSOLVER's column-major eigenvectors: row j = eigenvector j
    X[idx] = U[(long long)(first + k) * n + mu] / sqrt(s[first + k]);
}

__global__ void fock_kernel(const double* __restrict__ H, const double* __restrict__ J, const double* __restrict__ K,
                            long long len, double* __restrict__ F) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) F[i] = H[i] + J[i] - K[i];
}

// out[0] = sum D.*H, out[1] = sum D.*J, out[2] = sum D.*K (single block, deterministic)
__global__ void energy_kernel(const double* __restrict__ D, const double* __restrict__ H, const double* __restrict__ J,
                              const double* __restrict__ K, long long len, double* __restrict__ out) {
    double a = 0, b = 0, c = 0;
    for (long long i = threadIdx.x; i < len; i += blockDim.x) {
        const double d = D[i];
        a = fma(d, H[i], a);
        b = fma(d, J[i], b);
        c = fma(d, K[i], c);
    }
    __shared__ double sa[1024], sb[1024], sc[1024];
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sa[threadIdx.x] += sa[threadIdx.x + o];
            sb[threadIdx.x] += sb[threadIdx.x + o];
            sc[threadIdx.x] += sc[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sa[0];
        out[1] = sb[0];
        out[2] = sc[0];
    }
}

// E1 = T - T^T (n x n)
__global__ void antisym_kernel(const double* __restrict__ T, int n, double* __restrict__ E) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int i = (int)(idx / n), j = (int)(idx % n);
    E[idx] = T[idx] - T[(long long)j * n + i];
}

// out = max |x| (single block)
__global__ void absmax_kernel(const double* __restrict__ x, long long len, double* __restrict__ out) {
    double m = 0;
    for (long long i = threadIdx.x; i < len; i += blockDim.x) m = fmax(m, fabs(x[i]));
    __shared__ double sm[1024];
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

// DIIS: Bm[slot][j] = Bm[j][slot] = <e_slot, e_j> for the vectors present (one block per j)
__global__ void diis_dots_kernel(const double* __restrict__ E, long long len, int slot, const int* __restrict__ present,
                                 int size, double* __restrict__ Bm) {
    const int j = blockIdx.x;
    if (!present[j]) return;
    const double* a = E + (long long)slot * len;
    const double* b = E + (long long)j * len;
    double s = 0;
    for (long long i = threadIdx.x; i < len; i += blockDim.x) s = fma(a[i], b[i], s);
    __shared__ double sm[256];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        Bm[slot * DIIS_MAX + j] = sm[0];
        Bm[j * DIIS_MAX + slot] = sm[0];
    }
}

// Solve the Lagrange system [B -1; -1 0][c; l] = [0; -1] over the listed slots by Gaussian
// elimination with partial pivoting (single thread; m <= 16). coef[slot] receives c; status 0 ok,
// 1 singular (relative pivot below 1e-14).
__global__ void diis_solve_kernel(const double* __restrict__ Bm, const int* __restrict__ slots, int m,
                                  double* __restrict__ coef, int* __restrict__ status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double A[DIIS_MAX + 1][DIIS_MAX + 2];
    const int N = m + 1;
    double scale = 0;
    for (int i = 0; i < m; ++i) scale = fmax(scale, fabs(Bm[slots[i] * DIIS_MAX + slots[i]]));
    if (scale == 0) scale = 1;
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) A[i][j] = Bm[slots[i] * DIIS_MAX + slots[j]] / scale;
        A[i][m] = -1.0;
        A[i][N] = 0.0;
    }
    for (int j = 0; j < m; ++j) A[m][j] = -1.0;
    A[m][m] = 0.0;
    A[m][N] = -1.0;
    for (int col = 0; col < N; ++col) {
        int piv = col;
        for (int r = col + 1; r < N; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (fabs(A[piv][col]) < 1e-14) {
            *status = 1;
            return;
        }
        if (piv != col)
            for (int c = 0; c <= N; ++c) {
                double t = A[col][c];
                A[col][c] = A[piv][c];
                A[piv][c] = t;
            }
        for (int r = 0; r < N; ++r) {
            if (r == col) continue;
            const double f = A[r][col] / A[col][col];
            for (int c = col; c <= N; ++c) A[r][c] -= f * A[col][c];
        }
    }
    for (int i = 0; i < m; ++i) coef[slots[i]] = A[i][N] / A[i][i];
    *status = 0;
}

// Fx = sum_i coef[slot_i] F_slot_i
__global__ void diis_combine_kernel(const double* __restrict__ Fs, long long len, const int* __restrict__ slots, int m,
                                    const double* __restrict__ coef, double* __restrict__ Fx) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    double s = 0;
    for (int k = 0; k < m; ++k) s = fma(coef[slots[k]], Fs[(long long)slots[k] * len + i], s);
    Fx[i] = s;
}

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

struct Solver {
    df_handle* h;
    int n, nX;
    double* work = nullptr;
    int lwork = 0;
    int* info = nullptr;

    void eig(double* A, int m, double* w) {
        int lw = 0;
        DF_SOLVER(cusolverDnDsyevd_bufferSize(h->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, m, A, m, w, &lw));
        if (lw > lwork) {
            if (work) cudaFree(work);
            DF_CUDA(cudaMalloc((void**)&work, sizeof(double) * lw));
            lwork = lw;
        }
        DF_SOLVER(cusolverDnDsyevd(h->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, m, A, m, w, work, lwork, info));
        int hinfo = 0;
        DF_CUDA(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        DF_CUDA(cudaStreamSynchronize(h->stream));
        if (hinfo != 0) throw Error{DF_E_NUMERIC, "dsyevd failed, info " + std::to_string(hinfo)};
    }
    ~Solver() {
        if (work) cudaFree(work);
        if (info) cudaFree(info);
    }
};

}  // namespace

int scf_drive(df_handle* h, const df_options* o, df_result* r) {
    using clk = std::chrono::steady_clock;
    const auto t_start = clk::now();
    *r = df_result{};
    r->e_nuc = h->e_nuc;
    if (!h->built) {
        const auto t0 = clk::now();
        build_B(h, o->screen_tau, false);
        r->t_build_s = std::chrono::duration<double>(clk::now() - t0).count();
    }
    const int n = h->n, nocc = h->nocc;
    const long long nn = (long long)n * n;
    cudaStream_t s = h->stream;
    const int dsize = std::max(2, std::min(o->diis_size, DIIS_MAX));
    Solver sol{h, n, 0};
    DF_CUDA(cudaMalloc((void**)&sol.info, sizeof(int)));

    // --- orthogonaliser -------------------------------------------------------------------
    h->work1.alloc(nn);
    h->work2.alloc(nn);
    h->work3.alloc(nn);
    h->eps.alloc(n);
    DF_CUDA(cudaMemcpyAsync(h->work1.p, h->S.p, nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
    sol.eig(h->work1.p, n, h->eps.p);
    std::vector<double> sv(n);
    DF_CUDA(cudaMemcpy(sv.data(), h->eps.p, n * sizeof(double), cudaMemcpyDeviceToHost));
    int first = 0;
    while (first < n && sv[first] <= 1e-7) ++first;
    const int nX = n - first;
    if (nX < nocc) throw Error{DF_E_NUMERIC, "orthogonal basis smaller than the occupied space"};
    h->nX = nX;
    h->ndrop = first;
    r->n_dropped = first;
    h->X.alloc((size_t)n * nX);
    build_x_kernel<<<nblk((long long)n * nX), 256, 0, s>>>(h->work1.p, h->eps.p, n, first, nX, h->X.p);
    DF_CHECK_LAUNCH();

    h->F.alloc(nn);
    h->Fx.alloc(nn);
    h->Dm.alloc(nn);
    h->C.alloc((size_t)n * nX);
    DF_CUDA(cudaMemsetAsync(h->C.p, 0, sizeof(double) * n * nX, s));
    DF_CUDA(cudaMemsetAsync(h->eps.p, 0, sizeof(double) * n, s));
    ensure_jk_buffers(h, nocc);
    h->diisF.alloc((size_t)DIIS_MAX * nn);
    h->diisE.alloc((size_t)DIIS_MAX * nX * nX);
    h->diisB.alloc(DIIS_MAX * DIIS_MAX + 4 + DIIS_MAX);   // B matrix | energies(3) + maxerr | coef
    double* d_B = h->diisB.p;
    double* d_scal = d_B + DIIS_MAX * DIIS_MAX;
    double* d_coef = d_scal + 4;
    int* d_ints = nullptr;   // present[DIIS_MAX] | slots[DIIS_MAX] | status
    DF_CUDA(cudaMalloc((void**)&d_ints, sizeof(int) * (2 * DIIS_MAX + 1)));
    double* Fp = nullptr;    // X^T F X and its eigenvectors (nX x nX)
    DF_CUDA(cudaMalloc((void**)&Fp, sizeof(double) * nX * nX));
    double* T1 = nullptr;    // n x nX scratch
    DF_CUDA(cudaMalloc((void**)&T1, sizeof(double) * n * nX));

    auto roothaan = [&](const double* Fm) {
        // Fp = X^T F X ; eigenvectors ; C = X V ; D = 2 Cocc Cocc^T ; dC = Cocc (n x nocc)
        dgemm(s, false, false, n, nX, n, 1.0, Fm, n, h->X.p, nX, 0.0, T1, nX);
        dgemm(s, true, false, nX, nX, n, 1.0, h->X.p, nX, T1, nX, 0.0, Fp, nX);
        sol.eig(Fp, nX, h->eps.p);
        dgemm(s, false, true, n, nX, nX, 1.0, h->X.p, nX, Fp, nX, 0.0, h->C.p, nX);
        DF_CUDA(cudaMemcpy2DAsync(h->dC.p, sizeof(double) * nocc, h->C.p, sizeof(double) * nX, sizeof(double) * nocc, n,
                                  cudaMemcpyDeviceToDevice, s));
        dgemm(s, false, true, n, n, nocc, 2.0, h->dC.p, nocc, h->dC.p, nocc, 0.0, h->Dm.p, n);
    };

    int status = DF_E_NOTCONV;
    try {
        roothaan(h->H.p);   // core-Hamiltonian guess
        std::vector<int> present(DIIS_MAX, 0), order;
        std::vector<double> hs(4);
        double e_old = 0.0;
        double jk_ms = 0.0;
        cudaEvent_t ej0, ej1;
        DF_CUDA(cudaEventCreate(&ej0));
        DF_CUDA(cudaEventCreate(&ej1));
        const auto t_iter = clk::now();
        int it = 0;
        int slices = o->slices;   // split mode: o->slices early, SPLIT_LATE_SLICES once max|e| < SPLIT_RAMP_ERR
        for (it = 1; it <= o->max_iter; ++it) {
            DF_CUDA(cudaEventRecord(ej0, s));
            jk_dispatch(h, h->Dm.p, h->dC.p, nocc, h->dJ.p, h->dK.p, o->precision, slices);
            DF_CUDA(cudaEventRecord(ej1, s));
            fock_kernel<<<nblk(nn), 256, 0, s>>>(h->H.p, h->dJ.p, h->dK.p, nn, h->F.p);
            DF_CHECK_LAUNCH();
            energy_kernel<<<1, 1024, 0, s>>>(h->Dm.p, h->H.p, h->dJ.p, h->dK.p, nn, d_scal);
            DF_CHECK_LAUNCH();
            // error vector e = X^T (FDS - SDF) X
            dgemm(s, false, false, n, n, n, 1.0, h->F.p, n, h->Dm.p, n, 0.0, h->work1.p, n);
            dgemm(s, false, false, n, n, n, 1.0, h->work1.p, n, h->S.p, n, 0.0, h->work2.p, n);
            antisym_kernel<<<nblk(nn), 256, 0, s>>>(h->work2.p, n, h->work3.p);
            DF_CHECK_LAUNCH();
            dgemm(s, false, false, n, nX, n, 1.0, h->work3.p, n, h->X.p, nX, 0.0, T1, nX);
            // write e into the next DIIS slot directly
            int slot = 0;
            if ((int)order.size() < dsize) {
                while (present[slot]) ++slot;
            } else {
                slot = order.front();
                order.erase(order.begin());
                present[slot] = 0;
            }
            double* Eslot = h->diisE.p + (long long)slot * nX * nX;
            dgemm(s, true, false, nX, nX, n, 1.0, h->X.p, nX, T1, nX, 0.0, Eslot, nX);
            absmax_kernel<<<1, 1024, 0, s>>>(Eslot, (long long)nX * nX, d_scal + 3);
            DF_CHECK_LAUNCH();
            DF_CUDA(cudaMemcpyAsync(hs.data(), d_scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
            DF_CUDA(cudaStreamSynchronize(s));
            jk_ms += elapsed_ms(ej0, ej1);
            const double energy = hs[0] + 0.5 * hs[1] - 0.5 * hs[2] + h->e_nuc;
            const double err = hs[3];
            if (!std::isfinite(energy) || !std::isfinite(err)) {
                status = DF_E_NUMERIC;
                break;
            }
            r->energy = energy;
            r->e_one = hs[0];
            r->e_coul = 0.5 * hs[1];
            r->e_exch = -0.5 * hs[2];
            r->last_err = err;
            r->last_dE = (it > 1) ? energy - e_old : 0.0;
            r->iterations = it;
            const bool late_ready = o->precision != DF_PREC_SPLIT || slices >= SPLIT_LATE_SLICES;
            if (it > 1 && late_ready && std::fabs(energy - e_old) < o->conv_E && err < o->conv_err) {
                status = DF_OK;
                break;
            }
            bool ramp = false;
            if (o->precision == DF_PREC_SPLIT && slices < SPLIT_LATE_SLICES && err < SPLIT_RAMP_ERR) {
                slices = SPLIT_LATE_SLICES;
                r->ramp_iteration = it + 1;
                ramp = true;
            }
            e_old = energy;
            // DIIS bookkeeping: store F, dots, solve, combine. At the precision ramp the subspace is
            // restarted from the current Fock matrix: the earlier ones carry the coarser exchange.
            if (ramp) {
                for (int q : order) present[q] = 0;
                order.clear();
            }
            DF_CUDA(cudaMemcpyAsync(h->diisF.p + (long long)slot * nn, h->F.p, nn * sizeof(double),
                                    cudaMemcpyDeviceToDevice, s));
            present[slot] = 1;
            order.push_back(slot);
            DF_CUDA(cudaMemcpyAsync(d_ints, present.data(), sizeof(int) * DIIS_MAX, cudaMemcpyHostToDevice, s));
            diis_dots_kernel<<<DIIS_MAX, 256, 0, s>>>(h->diisE.p, (long long)nX * nX, slot, d_ints, DIIS_MAX, d_B);
            DF_CHECK_LAUNCH();
            const double* Fuse = h->F.p;
            while (it >= 2 && order.size() >= 2) {
                DF_CUDA(cudaMemcpyAsync(d_ints + DIIS_MAX, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, s));
                diis_solve_kernel<<<1, 1, 0, s>>>(d_B, d_ints + DIIS_MAX, (int)order.size(), d_coef, d_ints + 2 * DIIS_MAX);
                DF_CHECK_LAUNCH();
                int st = 0;
                DF_CUDA(cudaMemcpyAsync(&st, d_ints + 2 * DIIS_MAX, sizeof(int), cudaMemcpyDeviceToHost, s));
                DF_CUDA(cudaStreamSynchronize(s));
                if (st == 0) {
                    diis_combine_kernel<<<nblk(nn), 256, 0, s>>>(h->diisF.p, nn, d_ints + DIIS_MAX, (int)order.size(), d_coef,
                                                                h->Fx.p);
                    DF_CHECK_LAUNCH();
                    Fuse = h->Fx.p;
                    break;
                }
                present[order.front()] = 0;   // ill-conditioned: drop the oldest vector and retry
                order.erase(order.begin());
            }
            roothaan(Fuse);
        }
        if (it > o->max_iter) r->iterations = o->max_iter;
        r->t_iter_s = std::chrono::duration<double>(clk::now() - t_iter).count();
        r->t_jk_s = jk_ms / 1000.0;
        cudaEventDestroy(ej0);
        cudaEventDestroy(ej1);
    } catch (...) {
        cudaFree(d_ints);
        cudaFree(Fp);
        cudaFree(T1);
        throw;
    }
    cudaFree(d_ints);
    cudaFree(Fp);
    cudaFree(T1);
    r->converged = (status == DF_OK);
    r->status = status;
    r->t_total_s = std::chrono::duration<double>(clk::now() - t_start).count();
    return status;
}

}  // namespace dfhf
