// Restricted Hartree-Fock driver on the GPU (paper, section "Standard algorithms": RHF built on the
// density-fitted Fock builder). The paper gives no SCF details; this follows the textbook scheme:
//   canonical orthogonalisation X = U s^{-1/2} (eigenvalues of S below 1e-7 dropped),
//   core-Hamiltonian guess, F = H + J - K, E = tr(DH) + 1/2 tr(DJ) - 1/2 tr(DK) + E_nuc,
//   Pulay DIIS on e = X^T (F D S - S D F) X, Roothaan step X^T F X = V eps V^T, C = X V,
//   D = 2 C_occ C_occ^T (Aufbau), converged when |dE| < conv_E and max|e| < conv_err.
// DIIS works in the orthogonal basis: with F' = X^T F X and C = X V (so C^T S X = V^T), the error is
// e = 2 (F' P - P F') with P = V_occ V_occ^T, the extrapolation combines the F' of earlier iterations,
// and only the occupied orbitals C_occ = X V_occ are formed each iteration.
// Every step runs on the device in FP64 (DIIS included); only the energy and max|e| cross to the
// host each iteration for the convergence test. The symmetric eigensolver is cuSOLVER's dsyevd.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cmath>
#include <map>
#include <memory>
#include <set>
#include <thread>
#include <vector>

#include "common.cuh"

namespace dfhf {

void jk_dispatch(df_handle* h, const double* dD, const double* dC, int nocc, double* dJ, double* dK, int precision,
                 int slices);
void exchange_only(df_handle* h, const double* dC, int m, int precision, int slices, double* dK);

namespace {

constexpr int DIIS_MAX = 16;
constexpr int SPLIT_LATE_SLICES = 5;      // slices of the late split-precision exchange builds
constexpr double SPLIT_RAMP_ERR = 1e-4;   // max|e| below which the late builds start
constexpr int INC_SLICES = 3;             // slices of the density-change exchange builds (split mode)
constexpr int INC_RESET = 8;              // iterations per reference density (one full build, then changes)
constexpr int DIAG_RESET = 8;             // late iterations per full eigensolve when approximating the others

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

// E = a (T - T^T) (n x n)
__global__ void antisym_kernel(const double* __restrict__ T, int n, double a, double* __restrict__ E) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int i = (int)(idx / n), j = (int)(idx % n);
    E[idx] = a * (T[idx] - T[(long long)j * n + i]);
}

// E_slot = a (T - T^T) (n x n) into the DIIS slot held in device memory (a captured graph replays it)
__global__ void antisym_slot_kernel(const double* __restrict__ T, int n, double a, double* __restrict__ Ebase,
                                    const int* __restrict__ slot) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nn = (long long)n * n;
    if (idx >= nn) return;
    const int i = (int)(idx / n), j = (int)(idx % n);
    Ebase[(long long)*slot * nn + idx] = a * (T[idx] - T[(long long)j * n + i]);
}

// out = max |x_slot| over the DIIS slot held in device memory (single block)
__global__ void absmax_slot_kernel(const double* __restrict__ base, long long len, const int* __restrict__ slot,
                                   double* __restrict__ out) {
    const double* x = base + (long long)*slot * len;
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

// dst_slot = src (the Fock matrix of this iteration into the DIIS slot held in device memory)
__global__ void copy_to_slot_kernel(const double* __restrict__ src, double* __restrict__ base, long long len,
                                    const int* __restrict__ slot) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) base[(long long)*slot * len + i] = src[i];
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

// DIIS: Bm[slot][j] = Bm[j][slot] = <e_slot, e_j> for the vectors present (one block per j); vectors of
// len elements, `stride` apart
__global__ void diis_dots_kernel(const double* __restrict__ E, long long stride, long long len,
                                 const int* __restrict__ slotp, const int* __restrict__ present, int size,
                                 double* __restrict__ Bm) {
    const int j = blockIdx.x;
    const int slot = *slotp;
    if (!present[j]) return;
    const double* a = E + (long long)slot * stride;
    const double* b = E + (long long)j * stride;
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
// elimination with partial pivoting (single thread; m <= 16). coef[slot] receives c; status 0 ok.
// If a relative pivot falls below 1e-14 the system is singular: status 1 and coef selects the newest
// vector alone (plain F this iteration); the host then drops the oldest vector from the subspace.
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
            for (int i = 0; i < m; ++i) coef[slots[i]] = (i == m - 1) ? 1.0 : 0.0;
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

// Fx = sum_i coef[slot_i] F_slot_i (vectors of len elements, `stride` apart)
__global__ void diis_combine_kernel(const double* __restrict__ Fs, long long stride, long long len,
                                    const int* __restrict__ slots, int m, const double* __restrict__ coef,
                                    double* __restrict__ Fx) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    double s = 0;
    for (int k = 0; k < m; ++k) s = fma(coef[slots[k]], Fs[(long long)slots[k] * stride + i], s);
    Fx[i] = s;
}

// Incremental Fock build. With D = 2 C C^T and D_ref = 2 C_r C_r^T, the change is
// (D - D_ref)/2 = W G W^T, W = [C, C_r] (n x 2m), G = diag(+1 (m), -1 (m)). With W = Q R (QR) and the
// small eigenproblem R G R^T = Z L Z^T, (D - D_ref)/2 = sum_k l_k v_k v_k^T with v = Q Z; by Sylvester's
// law of inertia at most m of the l_k are positive and m negative, so in ascending order the first m
// carry the negative part and the last m the positive part. The exchange of the change is then
// K[C_+] - K[C_-] with C_+- = v sqrt(max(+-l, 0)) (the exchange here is the orbital form, K[C] = sum_P
// (B_P C)(B_P C)^T = sum_P B_P (D/2) B_P).

// W (column-major n x 2m) = [C, C_r] from two row-major n x m blocks
__global__ void assemble_w_kernel(const double* __restrict__ C, const double* __restrict__ Cr, int n, int m,
                                  double* __restrict__ W) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * 2 * m) return;
    const int j = (int)(idx / n), mu = (int)(idx % n);
    W[idx] = j < m ? C[(long long)mu * m + j] : Cr[(long long)mu * m + (j - m)];
}

// core = R G R^T (2m x 2m, symmetric) from the upper triangle R of a column-major QR factor (lda n)
__global__ void core_kernel(const double* __restrict__ W, int n, int m, double* __restrict__ core) {
    const int m2 = 2 * m;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m2 * m2) return;
    const int i = idx / m2, j = idx % m2;
    double s = 0;
    for (int k = max(i, j); k < m2; ++k) {
        const double t = W[(long long)k * n + i] * W[(long long)k * n + j];
        s += k < m ? t : -t;
    }
    core[idx] = s;
}

// Cm[mu][q] = v_q[mu] sqrt(max(-l_q, 0)), Cp[mu][q] = v_{m+q}[mu] sqrt(max(l_{m+q}, 0)); Vt rows are v_k
__global__ void split_factors_kernel(const double* __restrict__ Vt, const double* __restrict__ lam, int n, int m,
                                     double* __restrict__ Cp, double* __restrict__ Cm) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * m) return;
    const int mu = (int)(idx / m), q = (int)(idx % m);
    Cm[idx] = Vt[(long long)q * n + mu] * sqrt(fmax(-lam[q], 0.0));
    Cp[idx] = Vt[(long long)(m + q) * n + mu] * sqrt(fmax(lam[m + q], 0.0));
}

// K = Kref + Kp - Km
__global__ void k_update_kernel(const double* __restrict__ Kref, const double* __restrict__ Kp,
                                const double* __restrict__ Km, long long len, double* __restrict__ K) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) K[i] = Kref[i] + Kp[i] - Km[i];
}

// Approximate diagonalisation (Stewart, Csaszar and Pulay 1982): in the basis of the previous orbitals
// (occupied i, virtual a; energies eps from the last full eigensolve) the new Fock matrix has a small
// occupied-virtual block F'_ia; rotating by kappa_ia = F'_ia / (eps_a - eps_i) is the Roothaan step to
// first order: v_i <- v_i - sum_a kappa_ia v_a, v_a <- v_a + sum_i kappa_ia v_i.
__global__ void kappa_kernel(double* __restrict__ K, const double* __restrict__ eps, int nocc, int nvir) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nocc * nvir) return;
    const int i = (int)(idx / nvir), a = (int)(idx % nvir);
    K[idx] /= fmax(eps[nocc + a] - eps[i], 1e-3);
}

// P = (15/8) I - (5/4) M + (3/8) M^2: the series of M^{-1/2} about I to second order (M = Q Q^T near I)
__global__ void invsqrt_series_kernel(double* __restrict__ M, const double* __restrict__ M2, int m) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    M[idx] = (idx / m == idx % m ? 1.875 : 0.0) - 1.25 * M[idx] + 0.375 * M2[idx];
}

// c = a + b
__global__ void add_kernel2(const double* __restrict__ a, const double* __restrict__ b, long long len,
                            double* __restrict__ c) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) c[i] = a[i] + b[i];
}

// T = A^T (n x n)
__global__ void transpose_kernel(const double* __restrict__ A, int n, double* __restrict__ T) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int i = (int)(idx / n), j = (int)(idx % n);
    T[idx] = A[(long long)j * n + i];
}

// FP64 <-> FP32 copies (the mixed-precision eigensolve)
__global__ void to_float_kernel(const double* __restrict__ a, long long len, float* __restrict__ b) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) b[i] = (float)a[i];
}
__global__ void to_double_kernel(const float* __restrict__ a, long long len, double* __restrict__ b) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) b[i] = (double)a[i];
}

// a += b
__global__ void add_inplace_kernel(double* __restrict__ a, const double* __restrict__ b, long long len) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) a[i] += b[i];
}

// Vw[i][k] = V[i][k] w[i] for the first m rows (the occupied eigenvectors weighted by sqrt(n_i / 2))
__global__ void weight_rows_kernel(const double* __restrict__ V, const double* __restrict__ w, int m, int len,
                                   double* __restrict__ Vw) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)m * len) return;
    Vw[idx] = V[idx] * w[idx / len];
}

inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Occupations of orbitals with ascending energies eps: Aufbau in which a set of degenerate orbitals
// (energies within 1e-6 max(1, |eps|) of the set's first; a shell of l > 0 of a spherical atom) takes the
// electrons that reach it in equal shares of at most 2.
std::vector<double> aufbau_occupations(const std::vector<double>& eps, double nelec) {
    std::vector<double> occ(eps.size(), 0.0);
    double left = nelec;
    size_t i = 0;
    while (left > 0 && i < eps.size()) {
        size_t j = i + 1;
        while (j < eps.size() && std::fabs(eps[j] - eps[i]) <= 1e-6 * std::max(1.0, std::fabs(eps[i]))) ++j;
        const double take = std::min(left, 2.0 * (double)(j - i));
        for (size_t k = i; k < j; ++k) occ[k] = take / (double)(j - i);
        left -= take;
        i = j;
    }
    return occ;
}

namespace {

// Captured CUDA graphs of the SCF's repeated device sequences, one per kind of step (precision, slices,
// full or incremental exchange). A kind is launched directly the first time it occurs (buffers are sized and
// tile choices made then), captured from the stream the second time and replayed from then on; the sequence
// reads everything that changes between iterations (the DIIS slot) from device memory. A sequence that
// cannot be captured (a call that is not allowed in stream capture) is marked and launched directly;
// sequences that call cuSOLVER are not offered for capture at all.
class GraphCache {
  public:
    ~GraphCache() { clear(); }
    void clear() {
        for (auto& kv : exec_) cudaGraphExecDestroy(kv.second);
        exec_.clear();
        seen_.clear();
        broken_.clear();
    }
    template <typename F>
    void run(cudaStream_t s, int kind, F&& fn) {
        auto it = exec_.find(kind);
        if (it != exec_.end()) {
            DF_CUDA(cudaGraphLaunch(it->second, s));
            ++replays_;
            return;
        }
        if (!enabled_ || broken_.count(kind) || seen_[kind]++ == 0) {
            fn();
            return;
        }
        cudaGraph_t g = nullptr;
        DF_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        bool ok = true;
        try {
            fn();
        } catch (...) {
            ok = false;
        }
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        cudaGraphExec_t ex = nullptr;
        if (ok && e == cudaSuccess && g) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
        else ok = false;
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();   // a refused capture leaves no error for the next call
        if (!ok) {
            broken_.insert(kind);
            fn();   // nothing of the refused capture ran: launch the sequence directly
            return;
        }
        exec_[kind] = ex;
        DF_CUDA(cudaGraphLaunch(ex, s));
        ++replays_;
    }
    bool enabled_ = true;
    int replays_ = 0;

  private:
    std::map<int, cudaGraphExec_t> exec_;
    std::map<int, int> seen_;
    std::set<int> broken_;
};

// One molecule's SCF as a sequence of asynchronous iterations with a single host synchronisation each
// (the energy terms, max|e| and status words), so that many molecules can advance in lock-step on their
// own streams (scf_run_batch) while the GPU overlaps their kernels.
class ScfRun {
  public:
    ScfRun(df_handle* h, const df_options* o, df_result* r, const double* guess = nullptr)
        : h_(h), o_(*o), r_(r), guess_(guess) {}
    ~ScfRun() { release(); }

    // fractional occupations of nelec electrons by Aufbau with degenerate sets sharing equally (the atoms of
    // the SAD guess): the occupied rows of each Roothaan step are weighted by sqrt(n_i / 2), so that
    // D = 2 C_w C_w^T = sum n_i C_i C_i^T and the orbital-form exchange of C_w is half the exchange of D
    void set_fractional(double nelec) {
        frac_ = true;
        nelec_frac_ = nelec;
    }
    // the first Fock matrix from D0 = 2 C0 C0^T (C0: device, n x m, row-major), e.g. the SAD factor
    void set_initial_factor(const double* C0, int m) {
        C0_ = C0;
        m0_ = m;
    }
    const double* occupied_factor() const { return h_->dC.p; }
    int occupied_count() const { return nocc_; }

    // orthogonaliser and core-Hamiltonian guess (synchronises: the dropped-eigenvalue count is needed)
    void begin() {
        t_start_ = clk::now();
        *r_ = df_result{};
        r_->e_nuc = h_->e_nuc;
        if (!h_->built) {
            const auto t0 = clk::now();
            // FP64 precision: every step FP64, the whitening included; split: the tensor-core whitening
            build_B(h_, o_.screen_tau, false, o_.precision == DF_PREC_FP64 ? DF_WHITEN_FP64 : DF_WHITEN_SPLIT);
            r_->t_build_s = std::chrono::duration<double>(clk::now() - t0).count();
        }
        n_ = h_->n;
        nocc_ = h_->nocc;
        nn_ = (long long)n_ * n_;
        s_ = h_->stream;
        dsize_ = std::max(2, std::min(o_.diis_size, DIIS_MAX));
        slices_ = o_.slices;
        DF_CUDA(cudaMalloc((void**)&info_, sizeof(int)));
        DF_CUDA(cudaHostAlloc((void**)&pin_, sizeof(double) * 8, cudaHostAllocDefault));
        DF_CUDA(cudaHostAlloc((void**)&pin_ctl_, sizeof(int) * (2 * DIIS_MAX + 4), cudaHostAllocDefault));
        pin_ctl_[2 * DIIS_MAX + 2] = 0;
        pin_ctl_[2 * DIIS_MAX + 3] = 0;   // the DIIS slot of the iteration being built
        // per-phase timings take event synchronisations, which stream capture does not allow
        saved_sync_timing_ = h_->sync_timing;
        h_->sync_timing = false;
        const char* gv = std::getenv("DFHF_SCF_GRAPHS");
        graphs_.enabled_ = !frac_ && !(gv && gv[0] == '0');
        h_->tc_err_host = pin_ctl_ + 2 * DIIS_MAX + 2;   // timeout flag of the tensor-core kernels
        split_clear_error(h_);
        DF_CUDA(cudaEventCreate(&ev_done_));
        DF_CUDA(cudaEventCreate(&ej0_));
        DF_CUDA(cudaEventCreate(&ej1_));
        h_->work1.alloc(nn_);
        h_->work2.alloc(nn_);
        h_->work3.alloc(nn_);
        h_->eps.alloc(n_);
        DF_CUDA(cudaMemcpyAsync(h_->work1.p, h_->S.p, nn_ * sizeof(double), cudaMemcpyDeviceToDevice, s_));
        eig(h_->work1.p, n_, h_->eps.p);
        std::vector<double> sv(n_);
        DF_CUDA(cudaMemcpyAsync(sv.data(), h_->eps.p, n_ * sizeof(double), cudaMemcpyDeviceToHost, s_));
        int hinfo = 0;
        DF_CUDA(cudaMemcpyAsync(&hinfo, info_, sizeof(int), cudaMemcpyDeviceToHost, s_));
        DF_CUDA(cudaStreamSynchronize(s_));
        if (hinfo != 0) throw Error{DF_E_NUMERIC, "dsyevd of S failed, info " + std::to_string(hinfo)};
        int first = 0;
        while (first < n_ && sv[first] <= 1e-7) ++first;
        nX_ = n_ - first;
        if (nX_ < nocc_) throw Error{DF_E_NUMERIC, "orthogonal basis smaller than the occupied space"};
        h_->nX = nX_;
        h_->ndrop = first;
        r_->n_dropped = first;
        h_->X.alloc((size_t)n_ * nX_);
        build_x_kernel<<<nblk((long long)n_ * nX_), 256, 0, s_>>>(h_->work1.p, h_->eps.p, n_, first, nX_, h_->X.p);
        DF_CHECK_LAUNCH();
        h_->F.alloc(nn_);
        h_->Dm.alloc(nn_);
        h_->C.alloc((size_t)n_ * nX_);
        DF_CUDA(cudaMemsetAsync(h_->C.p, 0, sizeof(double) * n_ * nX_, s_));
        DF_CUDA(cudaMemsetAsync(h_->eps.p, 0, sizeof(double) * n_, s_));
        ensure_jk_buffers(h_, frac_ ? nX_ : std::max(nocc_, C0_ ? m0_ : 0));
        if (frac_) {
            DF_CUDA(cudaMalloc((void**)&vto_, sizeof(double) * ((long long)nX_ * nX_ + nX_)));
            wocc_ = vto_ + (long long)nX_ * nX_;
        }
        h_->diisF.alloc((size_t)DIIS_MAX * nn_);
        h_->diisE.alloc((size_t)DIIS_MAX * nX_ * nX_);
        h_->diisB.alloc(DIIS_MAX * DIIS_MAX + 8 + DIIS_MAX);   // B matrix | scalars (8) | coef
        d_B_ = h_->diisB.p;
        d_scal_ = d_B_ + DIIS_MAX * DIIS_MAX;
        d_coef_ = d_scal_ + 8;
        // present | slots | status | (unused) | slot of the iteration being built
        DF_CUDA(cudaMalloc((void**)&d_ints_, sizeof(int) * (2 * DIIS_MAX + 4)));
        DF_CUDA(cudaMemsetAsync(d_ints_, 0, sizeof(int) * (2 * DIIS_MAX + 4), s_));
        d_slot_ = d_ints_ + 2 * DIIS_MAX + 3;
        if (o_.incremental) alloc_reference();
        DF_CUDA(cudaMalloc((void**)&Fp_, sizeof(double) * nX_ * nX_));
        DF_CUDA(cudaMalloc((void**)&T1_, sizeof(double) * n_ * nX_));
        DF_CUDA(cudaMalloc((void**)&Fo_, sizeof(double) * nX_ * nX_));
        if (o_.approx_diag) {
            const long long no = nocc_, nv = nX_ - nocc_;
            DF_CUDA(cudaMalloc((void**)&abuf_, sizeof(double) * (3 * no * nX_ + no * nv + 2 * no * no)));
            DF_CUDA(cudaMalloc((void**)&f32a_, sizeof(float) * ((long long)nX_ * nX_ + nX_)));
            f32w_ = f32a_ + (long long)nX_ * nX_;
        }
        present_.assign(DIIS_MAX, 0);
        order_.clear();
        h_->history.clear();
        if (C0_) {
            // the first Fock matrix from the factor: C_occ = C0 (m0 columns), D = 2 C0 C0^T
            DF_CUDA(cudaMemcpyAsync(h_->dC.p, C0_, sizeof(double) * n_ * m0_, cudaMemcpyDeviceToDevice, s_));
            mm(s_, false, true, n_, n_, m0_, 2.0, h_->dC.p, m0_, h_->dC.p, m0_, 0.0, h_->Dm.p, n_);
            first_factor_ = true;
        } else if (guess_) {
            natural_orbitals(guess_);
        } else {
            to_orth(h_->H.p, Fp_);   // core-Hamiltonian guess
            solve_orth();
        }
        t_iter_ = clk::now();
        it_ = 0;
        done_ = false;
    }

    bool done() const { return done_; }

    // the enqueued iteration has completed on the device (errors of the stream are raised)
    bool ready() const {
        const cudaError_t e = cudaEventQuery(ev_done_);
        if (e == cudaSuccess) return true;
        if (e == cudaErrorNotReady) return false;
        DF_CUDA(e);
        return false;
    }

    // J/K, Fock, energy, error vector; scalars and status words copied to pinned memory; one event. The
    // host decisions come first; the device work of both parts is a captured graph per kind of step
    // (GraphCache), except in the iteration built from an initial factor.
    void enqueue_iteration() {
        ++it_;
        const bool inc = o_.incremental && late_ && inc_since_ref_ >= 0 && inc_since_ref_ + 1 < INC_RESET;
        const bool ref = !inc && o_.incremental && late_;
        slot_ = 0;
        if ((int)order_.size() < dsize_) {
            while (present_[slot_]) ++slot_;
        } else {
            slot_ = order_.front();
            order_.erase(order_.begin());
            present_[slot_] = 0;
        }
        pin_ctl_[2 * DIIS_MAX + 3] = slot_;
        DF_CUDA(cudaEventRecord(ej0_, s_));
        if (first_factor_) {
            if (m0_ > nocc_) first_factor_jk();
            else jk_dispatch(h_, h_->Dm.p, h_->dC.p, m0_, h_->dJ.p, h_->dK.p, o_.precision, slices_);
        } else if (inc) {
            // the incremental build calls cuSOLVER (QR and the small eigenproblem), which is not captured: a
            // refused capture left the solver unusable for the direct launch that follows
            jk_device(inc, ref);
        } else {
            const int kind = ((o_.precision == DF_PREC_SPLIT ? slices_ : 0) << 2) | (ref ? 1 : 0);
            graphs_.run(s_, kind, [&] { jk_device(inc, ref); });
        }
        if (inc) {
            ++inc_since_ref_;
            ++r_->incremental_builds;
        } else if (ref) {
            inc_since_ref_ = 0;
        }
        DF_CUDA(cudaEventRecord(ej1_, s_));
        if (first_factor_) {
            DF_CUDA(cudaMemcpyAsync(d_slot_, pin_ctl_ + 2 * DIIS_MAX + 3, sizeof(int), cudaMemcpyHostToDevice, s_));
            fock_kernel<<<nblk(nn_), 256, 0, s_>>>(h_->H.p, h_->dJ.p, h_->dK.p, nn_, h_->F.p);
            DF_CHECK_LAUNCH();
            energy_kernel<<<1, 1024, 0, s_>>>(h_->Dm.p, h_->H.p, h_->dJ.p, h_->dK.p, nn_, d_scal_);
            DF_CHECK_LAUNCH();
            to_orth(h_->F.p, Fo_);
            // the density is the factor's, not an Aufbau projector: e = X^T (F D S - S D F) X in full
            double* Eslot = h_->diisE.p + (long long)slot_ * nX_ * nX_;
            mm(s_, false, false, n_, n_, n_, 1.0, h_->F.p, n_, h_->Dm.p, n_, 0.0, h_->work1.p, n_);
            mm(s_, false, false, n_, n_, n_, 1.0, h_->work1.p, n_, h_->S.p, n_, 0.0, h_->work2.p, n_);
            antisym_kernel<<<nblk(nn_), 256, 0, s_>>>(h_->work2.p, n_, 1.0, h_->work3.p);
            DF_CHECK_LAUNCH();
            to_orth(h_->work3.p, Eslot);
            absmax_kernel<<<1, 1024, 0, s_>>>(Eslot, (long long)nX_ * nX_, d_scal_ + 3);
            DF_CHECK_LAUNCH();
            copy_scalars();
        } else {
            graphs_.run(s_, POST_KIND, [&] { post_device(); });
        }
        DF_CUDA(cudaEventRecord(ev_done_, s_));
    }

    // the exchange (and Coulomb) build of one iteration: full, full becoming the new reference, or K_ref
    // plus the exchange of the factorised density change
    void jk_device(bool inc, bool ref) {
        if (inc) {
            incremental_jk();
        } else {
            jk_dispatch(h_, h_->Dm.p, h_->dC.p, nocc_, h_->dJ.p, h_->dK.p, o_.precision, slices_);
            if (ref) set_reference();
        }
    }

    // Fock matrix, energy terms, F' = X^T F X and the error e = 2 (F' P - P F') (P = V_occ V_occ^T) into the
    // DIIS slot named in device memory, max|e|; scalars and status words to pinned memory
    void post_device() {
        DF_CUDA(cudaMemcpyAsync(d_slot_, pin_ctl_ + 2 * DIIS_MAX + 3, sizeof(int), cudaMemcpyHostToDevice, s_));
        fock_kernel<<<nblk(nn_), 256, 0, s_>>>(h_->H.p, h_->dJ.p, h_->dK.p, nn_, h_->F.p);
        DF_CHECK_LAUNCH();
        energy_kernel<<<1, 1024, 0, s_>>>(h_->Dm.p, h_->H.p, h_->dJ.p, h_->dK.p, nn_, d_scal_);
        DF_CHECK_LAUNCH();
        to_orth(h_->F.p, Fo_);
        mm(s_, false, true, nX_, nocc_, nX_, 1.0, Fo_, nX_, vt_, nX_, 0.0, h_->work2.p, nocc_);      // F' V_occ
        mm(s_, false, false, nX_, nX_, nocc_, 1.0, h_->work2.p, nocc_, vt_, nX_, 0.0, h_->work1.p, nX_);
        antisym_slot_kernel<<<nblk((long long)nX_ * nX_), 256, 0, s_>>>(h_->work1.p, nX_, 2.0, h_->diisE.p, d_slot_);
        DF_CHECK_LAUNCH();
        absmax_slot_kernel<<<1, 1024, 0, s_>>>(h_->diisE.p, (long long)nX_ * nX_, d_slot_, d_scal_ + 3);
        DF_CHECK_LAUNCH();
        copy_scalars();
    }

    void copy_scalars() {
        DF_CUDA(cudaMemcpyAsync(pin_, d_scal_, 4 * sizeof(double), cudaMemcpyDeviceToHost, s_));
        DF_CUDA(cudaMemcpyAsync(pin_ctl_ + 2 * DIIS_MAX, d_ints_ + 2 * DIIS_MAX, sizeof(int), cudaMemcpyDeviceToHost, s_));
        DF_CUDA(cudaMemcpyAsync(pin_ctl_ + 2 * DIIS_MAX + 1, info_, sizeof(int), cudaMemcpyDeviceToHost, s_));
    }

    // wait for the iteration, test convergence; if not done, enqueue DIIS and the Roothaan step
    void finish_iteration() {
        DF_CUDA(cudaEventSynchronize(ev_done_));
        const double this_jk = elapsed_ms(ej0_, ej1_);
        jk_ms_ += this_jk;
        if (pin_ctl_[2 * DIIS_MAX + 1] != 0)
            throw Error{DF_E_NUMERIC, "dsyevd failed, info " + std::to_string(pin_ctl_[2 * DIIS_MAX + 1])};
        if (pin_ctl_[2 * DIIS_MAX + 2] != 0)
            throw Error{DF_E_TIMEOUT, "tensor-core exchange kernel timed out waiting on a barrier"};
        if (pin_ctl_[2 * DIIS_MAX] != 0 && !order_.empty()) {   // last DIIS system was singular
            const int old = order_.front();
            if (old != slot_) {
                present_[old] = 0;
                order_.erase(order_.begin());
            }
        }
        const double energy = pin_[0] + 0.5 * pin_[1] - 0.5 * pin_[2] + h_->e_nuc;
        const double err = pin_[3];
        h_->history.insert(h_->history.end(), {(double)it_, energy, it_ > 1 ? energy - e_old_ : 0.0, err,
                                               o_.precision == DF_PREC_SPLIT ? (double)slices_ : 0.0, this_jk});
        if (!std::isfinite(energy) || !std::isfinite(err)) {
            status_ = DF_E_NUMERIC;
            return finish();
        }
        r_->energy = energy;
        r_->e_one = pin_[0];
        r_->e_coul = 0.5 * pin_[1];
        r_->e_exch = -0.5 * pin_[2];
        r_->last_err = err;
        r_->last_dE = (it_ > 1) ? energy - e_old_ : 0.0;
        r_->iterations = it_;
        const bool late_ready = o_.precision != DF_PREC_SPLIT || slices_ >= SPLIT_LATE_SLICES;
        if (it_ > 1 && late_ready && std::fabs(energy - e_old_) < o_.conv_E && err < o_.conv_err) {
            status_ = DF_OK;
            return finish();
        }
        if (it_ >= o_.max_iter) {
            status_ = DF_E_NOTCONV;
            return finish();
        }
        e_old_ = energy;
        bool ramp = false;
        if (o_.precision == DF_PREC_SPLIT && slices_ < SPLIT_LATE_SLICES && err < SPLIT_RAMP_ERR) {
            slices_ = SPLIT_LATE_SLICES;
            r_->ramp_iteration = it_ + 1;
            ramp = true;
        }
        if (!late_ && err < SPLIT_RAMP_ERR) late_ = true;
        // DIIS: at the precision ramp the subspace restarts from the current Fock matrix (the earlier
        // ones carry the coarser exchange)
        if (ramp) {
            for (int q : order_) present_[q] = 0;
            order_.clear();
        }
        const long long no = (long long)nX_ * nX_;
        copy_to_slot_kernel<<<nblk(no), 256, 0, s_>>>(Fo_, h_->diisF.p, no, d_slot_);
        DF_CHECK_LAUNCH();
        present_[slot_] = 1;
        order_.push_back(slot_);
        for (int q = 0; q < DIIS_MAX; ++q) pin_ctl_[q] = present_[q];
        for (size_t q = 0; q < order_.size(); ++q) pin_ctl_[DIIS_MAX + q] = order_[q];
        DF_CUDA(cudaMemcpyAsync(d_ints_, pin_ctl_, sizeof(int) * 2 * DIIS_MAX, cudaMemcpyHostToDevice, s_));
        diis_dots_kernel<<<DIIS_MAX, 256, 0, s_>>>(h_->diisE.p, (long long)nX_ * nX_, (long long)nX_ * nX_, d_slot_,
                                                   d_ints_, DIIS_MAX, d_B_);
        DF_CHECK_LAUNCH();
        // Roothaan step: a full eigensolve, or late (options.approx_diag) a rotation of the previous
        // orbitals, with a full eigensolve every DIAG_RESET late iterations
        const bool approx = o_.approx_diag && late_ && fock_basis_ && nX_ > nocc_ && diag_since_full_ >= 0 &&
                            diag_since_full_ + 1 < DIAG_RESET;
        double* Fx = approx ? h_->work3.p : Fp_;
        if (it_ >= 2 && order_.size() >= 2) {
            diis_solve_kernel<<<1, 1, 0, s_>>>(d_B_, d_ints_ + DIIS_MAX, (int)order_.size(), d_coef_,
                                               d_ints_ + 2 * DIIS_MAX);
            DF_CHECK_LAUNCH();
            diis_combine_kernel<<<nblk(no), 256, 0, s_>>>(h_->diisF.p, no, no, d_ints_ + DIIS_MAX, (int)order_.size(),
                                                         d_coef_, Fx);
            DF_CHECK_LAUNCH();
        } else {
            DF_CUDA(cudaMemsetAsync(d_ints_ + 2 * DIIS_MAX, 0, sizeof(int), s_));
            DF_CUDA(cudaMemcpyAsync(Fx, Fo_, no * sizeof(double), cudaMemcpyDeviceToDevice, s_));
        }
        if (approx) {
            approx_orth(Fx);
            ++diag_since_full_;
            ++r_->approx_steps;
        } else {
            solve_orth();
            if (late_) diag_since_full_ = 0;
        }
        first_factor_ = false;
        last_approx_ = approx || mixed_step_;
    }

    int status() const { return status_; }

  private:
    using clk = std::chrono::steady_clock;

    // SCF algebra products (X^T F X, the DIIS error, the orbital and density products, the approximate
    // diagonalisation) are FP64 in both precision modes: only the exchange contraction is split
    void mm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
            const double* B, int ldb, double beta, double* C, int ldc) {
        dgemm(s, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    }

    // J and K of the first Fock matrix from the factor C0 (m0 > nocc columns): J from D0, K as the sum of the
    // exchanges of column blocks of at most nocc columns (the orbital-form exchange is additive over columns),
    // so the exchange buffers keep the width of the occupied orbitals
    void first_factor_jk() {
        coulomb_fp64(h_, h_->Dm.p, h_->dJ.p);
        const int m1 = nocc_, m2 = m0_ - nocc_;
        double* Ca = h_->work1.p;   // n x m1
        double* Cb = h_->work2.p;   // n x m2 (m0 <= n: both fit an n x n buffer)
        DF_CUDA(cudaMemcpy2DAsync(Ca, sizeof(double) * m1, h_->dC.p, sizeof(double) * m0_, sizeof(double) * m1, n_,
                                  cudaMemcpyDeviceToDevice, s_));
        DF_CUDA(cudaMemcpy2DAsync(Cb, sizeof(double) * m2, h_->dC.p + m1, sizeof(double) * m0_, sizeof(double) * m2, n_,
                                  cudaMemcpyDeviceToDevice, s_));
        exchange_only(h_, Ca, m1, o_.precision, slices_, h_->dK.p);
        exchange_only(h_, Cb, m2, o_.precision, slices_, h_->work3.p);
        add_inplace_kernel<<<nblk(nn_), 256, 0, s_>>>(h_->dK.p, h_->work3.p, nn_);
        DF_CHECK_LAUNCH();
    }

    // buffers of the incremental Fock build
    void alloc_reference() {
        const long long m = nocc_;
        DF_CUDA(cudaMalloc((void**)&Kref_, sizeof(double) * nn_ * 3));   // K_ref | K_+ | K_-
        DF_CUDA(cudaMalloc((void**)&Cref_, sizeof(double) * n_ * m * 3));   // C_ref | C_+ | C_-
        DF_CUDA(cudaMalloc((void**)&Wq_, sizeof(double) * n_ * 2 * m * 2));   // W / Q | V^T
        DF_CUDA(cudaMalloc((void**)&core_, sizeof(double) * (4 * m * m + 4 * m)));   // core | l | tau
    }

    // the full build just enqueued becomes the reference: K_ref = K, C_ref = C_occ
    void set_reference() {
        DF_CUDA(cudaMemcpyAsync(Kref_, h_->dK.p, nn_ * sizeof(double), cudaMemcpyDeviceToDevice, s_));
        DF_CUDA(cudaMemcpyAsync(Cref_, h_->dC.p, sizeof(double) * n_ * nocc_, cudaMemcpyDeviceToDevice, s_));
    }

    // J in full; K = K_ref + K[C_+] - K[C_-] from the factorised density change
    void incremental_jk() {
        const int m = nocc_, m2 = 2 * nocc_;
        ensure_jk_buffers(h_, nocc_);
        coulomb_fp64(h_, h_->Dm.p, h_->dJ.p);
        double* W = Wq_;
        double* Vt = Wq_ + (long long)n_ * m2;
        double* lam = core_ + (long long)m2 * m2;
        double* tau = lam + m2;
        double *Cp = Cref_ + (long long)n_ * m, *Cm = Cp + (long long)n_ * m;
        double *Kp = Kref_ + nn_, *Km = Kp + nn_;
        assemble_w_kernel<<<nblk((long long)n_ * m2), 256, 0, s_>>>(h_->dC.p, Cref_, n_, m, W);
        DF_CHECK_LAUNCH();
        int lw = 0, lw2 = 0;
        DF_SOLVER(cusolverDnDgeqrf_bufferSize(h_->solver, n_, m2, W, n_, &lw));
        DF_SOLVER(cusolverDnDorgqr_bufferSize(h_->solver, n_, m2, m2, W, n_, tau, &lw2));
        grow_work(std::max(lw, lw2));
        DF_SOLVER(cusolverDnDgeqrf(h_->solver, n_, m2, W, n_, tau, work_, lwork_, info_));
        core_kernel<<<nblk((long long)m2 * m2), 256, 0, s_>>>(W, n_, m, core_);
        DF_CHECK_LAUNCH();
        DF_SOLVER(cusolverDnDorgqr(h_->solver, n_, m2, m2, W, n_, tau, work_, lwork_, info_));
        eig(core_, m2, lam);
        // V^T (2m x n): row k = sum_j Z[k][j] Q[:, j]; Q column-major n x 2m is the row-major 2m x n Q^T
        mm(s_, false, false, m2, n_, m2, 1.0, core_, m2, W, n_, 0.0, Vt, n_);
        split_factors_kernel<<<nblk((long long)n_ * m), 256, 0, s_>>>(Vt, lam, n_, m, Cp, Cm);
        DF_CHECK_LAUNCH();
        const int inc_slices = o_.precision == DF_PREC_SPLIT ? INC_SLICES : 0;
        exchange_only(h_, Cp, m, o_.precision, inc_slices, Kp);
        exchange_only(h_, Cm, m, o_.precision, inc_slices, Km);
        k_update_kernel<<<nblk(nn_), 256, 0, s_>>>(Kref_, Kp, Km, nn_, h_->dK.p);
        DF_CHECK_LAUNCH();
    }

    void grow_work(int lw) {
        if (lw > lwork_) {
            if (work_) cudaFree(work_);
            work_ = nullptr;
            DF_CUDA(cudaMalloc((void**)&work_, sizeof(double) * lw));
            lwork_ = lw;
        }
    }

    void eig(double* A, int m, double* w) {
        int lw = 0;
        DF_SOLVER(cusolverDnDsyevd_bufferSize(h_->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, m, A, m, w, &lw));
        grow_work(lw);
        DF_SOLVER(cusolverDnDsyevd(h_->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, m, A, m, w, work_,
                                   lwork_, info_));
    }

    // Fo = X^T Fm X (nX x nX)
    void to_orth(const double* Fm, double* Fo) {
        mm(s_, false, false, n_, nX_, n_, 1.0, Fm, n_, h_->X.p, nX_, 0.0, T1_, nX_);
        mm(s_, true, false, nX_, nX_, n_, 1.0, h_->X.p, nX_, T1_, nX_, 0.0, Fo, nX_);
    }

    // Roothaan step on the orthogonal-basis Fock matrix held in Fp_: eigenvectors in place (row j of the
    // row-major view is eigenvector j, ascending), the nocc lowest occupied. With options.approx_diag (and
    // integer occupations) the eigensolve is FP32 (cuSOLVER's FP64 eigensolver takes 3-4x longer at
    // n = 1600-2000 and holds the host thread while it runs) and is refined against the FP64 matrix by one
    // rotation of the occupied-virtual block and the re-orthonormalisation of approx_orth: the FP32
    // eigenvectors' errors (about 1e-6) enter the occupied space at second order, and the virtual rows are
    // projected out of the occupied space. The orbital energies keep FP32 accuracy (they only scale the
    // rotations); the final orbitals and energies are refreshed in FP64 when the run ends.
    void solve_orth() {
        if (o_.approx_diag && !frac_ && nX_ > nocc_) {
            const long long no = (long long)nX_ * nX_;
            DF_CUDA(cudaMemcpyAsync(h_->work3.p, Fp_, sizeof(double) * no, cudaMemcpyDeviceToDevice, s_));
            to_float_kernel<<<nblk(no), 256, 0, s_>>>(Fp_, no, f32a_);
            DF_CHECK_LAUNCH();
            int lw = 0;
            DF_SOLVER(cusolverDnSsyevd_bufferSize(h_->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, nX_, f32a_,
                                                  nX_, f32w_, &lw));
            if (lw > f32lwork_) {
                if (f32work_) cudaFree(f32work_);
                f32work_ = nullptr;
                DF_CUDA(cudaMalloc((void**)&f32work_, sizeof(float) * lw));
                f32lwork_ = lw;
            }
            DF_SOLVER(cusolverDnSsyevd(h_->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, nX_, f32a_, nX_,
                                       f32w_, f32work_, f32lwork_, info_));
            to_double_kernel<<<nblk(no), 256, 0, s_>>>(f32a_, no, Fp_);
            DF_CHECK_LAUNCH();
            to_double_kernel<<<nblk(nX_), 256, 0, s_>>>(f32w_, nX_, h_->eps.p);
            DF_CHECK_LAUNCH();
            fock_basis_ = true;
            approx_orth(h_->work3.p);
            // the virtual rows made exactly orthogonal to the refined occupied rows: FP32 rows are orthogonal
            // only to about 1e-7, and the late rotations, whose stationarity condition is F'_ia = 0 over these
            // rows, would otherwise stop at a commutator floor of that order times |F|
            const int nocc = nocc_, nv = nX_ - nocc_;
            double* Vo = Fp_;
            double* Vv = Fp_ + (long long)nocc * nX_;
            double* O = h_->work1.p;   // nv x nocc
            mm(s_, false, true, nv, nocc, nX_, 1.0, Vv, nX_, Vo, nX_, 0.0, O, nocc);
            mm(s_, false, false, nv, nX_, nocc, -1.0, O, nocc, Vo, nX_, 1.0, Vv, nX_);
            mixed_step_ = true;
            return;
        }
        mixed_step_ = false;
        eig(Fp_, nX_, h_->eps.p);
        vt_ = Fp_;
        fock_basis_ = true;
        if (frac_) weight_occupied();
        occupy();
    }

    // fractional mode: occupations from the new orbital energies (read back: the atoms are small), the
    // occupied eigenvectors weighted by sqrt(n_i / 2) into vto_
    void weight_occupied() {
        std::vector<double> eps(nX_);
        DF_CUDA(cudaMemcpyAsync(eps.data(), h_->eps.p, sizeof(double) * nX_, cudaMemcpyDeviceToHost, s_));
        DF_CUDA(cudaStreamSynchronize(s_));
        const std::vector<double> occ = aufbau_occupations(eps, nelec_frac_);
        occ_w_.assign(nX_, 0.0);
        int m = 0;
        for (int i = 0; i < nX_; ++i)
            if (occ[i] > 0) {
                occ_w_[i] = std::sqrt(occ[i] / 2.0);
                m = i + 1;
            }
        if (m == 0) throw Error{DF_E_NUMERIC, "fractional occupation: no occupied orbital"};
        nocc_ = m;
        DF_CUDA(cudaMemcpyAsync(wocc_, occ_w_.data(), sizeof(double) * nX_, cudaMemcpyHostToDevice, s_));
        weight_rows_kernel<<<nblk((long long)m * nX_), 256, 0, s_>>>(Fp_, wocc_, m, nX_, vto_);
        DF_CHECK_LAUNCH();
        DF_CUDA(cudaStreamSynchronize(s_));   // occ_w_ is read by the copy above
        vt_ = vto_;
    }

    // approximate Roothaan step on the orthogonal-basis Fock matrix Fx: the rows of Fp_ (occupied first)
    // rotated by kappa, the occupied rows re-orthonormalised by two rounds of the inverse-square-root
    // series; the virtual rows keep first-order accuracy until the next full eigensolve
    void approx_orth(const double* Fx) {
        const int no = nocc_, nv = nX_ - nocc_;
        double* Vo = Fp_;
        double* Vv = Fp_ + (long long)no * nX_;
        double* G = abuf_;                          // no x nX
        double* Kp = G + (long long)no * nX_;       // no x nv
        double* VoN = Kp + (long long)no * nv;      // no x nX
        double* Q = VoN + (long long)no * nX_;      // no x nX
        double* M = Q + (long long)no * nX_;        // no x no
        double* M2 = M + (long long)no * no;        // no x no
        double* VvN = h_->work1.p;                  // nv x nX
        mm(s_, false, false, no, nX_, nX_, 1.0, Vo, nX_, Fx, nX_, 0.0, G, nX_);
        mm(s_, false, true, no, nv, nX_, 1.0, G, nX_, Vv, nX_, 0.0, Kp, nv);    // F'_ia
        kappa_kernel<<<nblk((long long)no * nv), 256, 0, s_>>>(Kp, h_->eps.p, no, nv);
        DF_CHECK_LAUNCH();
        DF_CUDA(cudaMemcpyAsync(VoN, Vo, sizeof(double) * no * nX_, cudaMemcpyDeviceToDevice, s_));
        DF_CUDA(cudaMemcpyAsync(VvN, Vv, sizeof(double) * nv * nX_, cudaMemcpyDeviceToDevice, s_));
        mm(s_, false, false, no, nX_, nv, -1.0, Kp, nv, Vv, nX_, 1.0, VoN, nX_);
        mm(s_, true, false, nv, nX_, no, 1.0, Kp, nv, Vo, nX_, 1.0, VvN, nX_);
        double *src = VoN, *dst = Q;
        for (int round = 0; round < 2; ++round) {
            mm(s_, false, true, no, no, nX_, 1.0, src, nX_, src, nX_, 0.0, M, no);
            mm(s_, false, false, no, no, no, 1.0, M, no, M, no, 0.0, M2, no);
            invsqrt_series_kernel<<<nblk((long long)no * no), 256, 0, s_>>>(M, M2, no);
            DF_CHECK_LAUNCH();
            mm(s_, false, false, no, nX_, no, 1.0, M, no, src, nX_, 0.0, dst, nX_);
            std::swap(src, dst);
        }
        DF_CUDA(cudaMemcpyAsync(Vo, src, sizeof(double) * no * nX_, cudaMemcpyDeviceToDevice, s_));
        DF_CUDA(cudaMemcpyAsync(Vv, VvN, sizeof(double) * nv * nX_, cudaMemcpyDeviceToDevice, s_));
        vt_ = Fp_;
        occupy();
    }

    // dC = C_occ = X V_occ (n x nocc) from the occupied rows vt_ ; D = 2 C_occ C_occ^T
    void occupy() {
        mm(s_, false, true, n_, nocc_, nX_, 1.0, h_->X.p, nX_, vt_, nX_, 0.0, h_->dC.p, nocc_);
        mm(s_, false, true, n_, n_, nocc_, 2.0, h_->dC.p, nocc_, h_->dC.p, nocc_, 0.0, h_->Dm.p, n_);
    }

    // first orbitals from a guess density D0 (host): the nocc eigenvectors of X^T S D0 S X with the
    // largest eigenvalues, C = X V_occ, D = 2 C C^T
    void natural_orbitals(const double* D0) {
        DF_CUDA(cudaMemcpyAsync(h_->work3.p, D0, nn_ * sizeof(double), cudaMemcpyHostToDevice, s_));
        mm(s_, false, false, n_, n_, n_, 1.0, h_->S.p, n_, h_->work3.p, n_, 0.0, h_->work1.p, n_);
        mm(s_, false, false, n_, n_, n_, 1.0, h_->work1.p, n_, h_->S.p, n_, 0.0, h_->work2.p, n_);
        mm(s_, false, false, n_, nX_, n_, 1.0, h_->work2.p, n_, h_->X.p, nX_, 0.0, T1_, nX_);
        mm(s_, true, false, nX_, nX_, n_, 1.0, h_->X.p, nX_, T1_, nX_, 0.0, Fp_, nX_);
        eig(Fp_, nX_, h_->eps.p);
        fock_basis_ = false;
        // ascending eigenvalues: the occupied natural orbitals are the last nocc eigenvectors
        vt_ = Fp_ + (long long)(nX_ - nocc_) * nX_;
        occupy();
        DF_CUDA(cudaStreamSynchronize(s_));   // D0 is host memory owned by the caller
    }

    void finish() {
        h_->tc_err_host = nullptr;
        // after an approximate step the orbital energies and virtual orbitals are refreshed from the last
        // Fock matrix; then all orbitals of the last Roothaan step, C = X V
        if (last_approx_) {
            DF_CUDA(cudaMemcpyAsync(Fp_, Fo_, sizeof(double) * nX_ * nX_, cudaMemcpyDeviceToDevice, s_));
            eig(Fp_, nX_, h_->eps.p);
        }
        if (vt_ == Fp_) mm(s_, false, true, n_, nX_, nX_, 1.0, h_->X.p, nX_, Fp_, nX_, 0.0, h_->C.p, nX_);
        done_ = true;
        r_->converged = (status_ == DF_OK);
        r_->status = status_;
        r_->t_iter_s = std::chrono::duration<double>(clk::now() - t_iter_).count();
        r_->t_jk_s = jk_ms_ / 1000.0;
        r_->t_total_s = std::chrono::duration<double>(clk::now() - t_start_).count();
        r_->graph_launches = graphs_.replays_;
    }

    void release() {
        // work this run queued (on an error path: copies into the pinned words, kernels on its buffers)
        // completes before anything is freed
        if (s_) cudaStreamSynchronize(s_);
        graphs_.clear();
        if (pin_ctl_ && h_) h_->sync_timing = saved_sync_timing_;
        if (h_ && pin_ctl_ && h_->tc_err_host == pin_ctl_ + 2 * DIIS_MAX + 2) h_->tc_err_host = nullptr;
        if (work_) cudaFree(work_);
        if (info_) cudaFree(info_);
        if (d_ints_) cudaFree(d_ints_);
        if (Fp_) cudaFree(Fp_);
        if (T1_) cudaFree(T1_);
        if (Fo_) cudaFree(Fo_);
        if (abuf_) cudaFree(abuf_);
        abuf_ = nullptr;
        if (f32a_) cudaFree(f32a_);
        if (f32work_) cudaFree(f32work_);
        f32a_ = f32w_ = f32work_ = nullptr;
        f32lwork_ = 0;
        if (vto_) cudaFree(vto_);
        vto_ = wocc_ = nullptr;
        if (Kref_) cudaFree(Kref_);
        if (Cref_) cudaFree(Cref_);
        if (Wq_) cudaFree(Wq_);
        if (core_) cudaFree(core_);
        Kref_ = Cref_ = Wq_ = core_ = nullptr;
        if (pin_) cudaFreeHost(pin_);
        if (pin_ctl_) cudaFreeHost(pin_ctl_);
        if (ev_done_) cudaEventDestroy(ev_done_);
        if (ej0_) cudaEventDestroy(ej0_);
        if (ej1_) cudaEventDestroy(ej1_);
        work_ = nullptr;
        info_ = nullptr;
        d_ints_ = nullptr;
        Fp_ = T1_ = Fo_ = nullptr;
        pin_ = nullptr;
        pin_ctl_ = nullptr;
        ev_done_ = ej0_ = ej1_ = nullptr;
    }

    df_handle* h_;
    df_options o_;
    df_result* r_;
    const double* guess_ = nullptr;
    clk::time_point t_start_, t_iter_;
    int n_ = 0, nocc_ = 0, nX_ = 0, dsize_ = 2, slices_ = 0, it_ = 0, slot_ = 0;
    long long nn_ = 0;
    cudaStream_t s_ = nullptr;
    double* work_ = nullptr;
    int lwork_ = 0;
    int* info_ = nullptr;
    int* d_ints_ = nullptr;
    double *d_B_ = nullptr, *d_scal_ = nullptr, *d_coef_ = nullptr, *Fp_ = nullptr, *T1_ = nullptr, *Fo_ = nullptr;
    const double* vt_ = nullptr;   // occupied eigenvectors (nocc rows of length nX) of the last Roothaan step
    double *Kref_ = nullptr, *Cref_ = nullptr, *Wq_ = nullptr, *core_ = nullptr;   // incremental Fock state
    bool late_ = false;            // past the max|e| < 1e-4 point (split: the 5-slice builds)
    double* abuf_ = nullptr;       // approximate diagonalisation scratch
    float *f32a_ = nullptr, *f32w_ = nullptr, *f32work_ = nullptr;   // FP32 eigensolve: matrix, values, workspace
    int f32lwork_ = 0;
    bool mixed_step_ = false;      // the last full Roothaan step was the FP32 eigensolve with FP64 refinement
    bool fock_basis_ = false;      // Fp_ holds eigenvectors of a Fock matrix (eps their energies)
    bool last_approx_ = false;     // the last Roothaan step was approximate
    int diag_since_full_ = -1;     // late approximate steps since the last full eigensolve (-1: none yet)
    int inc_since_ref_ = -1;       // density-change builds since the reference (-1: no reference yet)
    double* pin_ = nullptr;
    int* pin_ctl_ = nullptr;
    cudaEvent_t ev_done_ = nullptr, ej0_ = nullptr, ej1_ = nullptr;
    std::vector<int> present_, order_;
    double e_old_ = 0.0, jk_ms_ = 0.0;
    bool done_ = false;
    int status_ = DF_E_NOTCONV;
    bool frac_ = false;            // fractional occupations (set_fractional)
    double nelec_frac_ = 0.0;
    double* vto_ = nullptr;        // weighted occupied rows (fractional mode) | their weights (wocc_)
    double* wocc_ = nullptr;
    std::vector<double> occ_w_;
    const double* C0_ = nullptr;   // initial factor (set_initial_factor): the first Fock matrix from 2 C0 C0^T
    int m0_ = 0;
    bool first_factor_ = false;    // the iteration being built uses C0 (no Roothaan step taken yet)
    static constexpr int POST_KIND = 1 << 10;   // graph kind of the post-J/K part
    GraphCache graphs_;
    int* d_slot_ = nullptr;        // device copy of the DIIS slot of the iteration being built
    bool saved_sync_timing_ = true;
};

// Unrestricted Hartree-Fock (paper, section "Program features", "Standard algorithms": UHF on the
// density-fitted Fock builder). Spin densities D_s = C_s C_s^T (no factor 2); J from D_a + D_b (eq. 3);
// K_s = sum_{P,i in s} Y Y^T from the spin's occupied orbitals (eqs. 1-2, first forms; FP64 or split
// precision, the split form at 3 slices until max|e| < 1e-4 and 5 slices after, converging only on the
// 5-slice builds); F_s = H + J - K_s; E = 1/2 tr(D_a (H + F_a)) + 1/2 tr(D_b (H + F_b)) + E_nuc. Pulay DIIS
// over the stacked pair (F'_a, F'_b) with errors F'_s P_s - P_s F'_s (P_s = V_s,occ V_s,occ^T; the
// orthogonal-basis form of X^T (F_s D_s S - S D_s F_s) X), one set of coefficients for both spins;
// core-Hamiltonian start for both spins, or (options.guess = DF_GUESS_SPIN) the natural orbitals of the
// spin densities of the handle's last open-shell run; every step on the device in FP64 except the exchange
// contraction.

// Restricted open-shell effective Fock matrix in the basis of the current orbitals (closed p < nb, open
// nb <= p < na, virtual p >= na): closed-open pairs take F_b, open-virtual pairs F_a, all others
// (F_a + F_b) / 2. Fa_mo becomes the effective matrix plus the level shift (lambda on the virtual,
// lambda / 2 on the open diagonal), Fb_mo its off-diagonal class blocks (the DIIS error).
__global__ void rohf_effective_kernel(double* __restrict__ Fa_mo, double* __restrict__ Fb_mo, int m, int na, int nb,
                                      double shift) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)m * m) return;
    const int p = (int)(idx / m), q = (int)(idx % m);
    const int cp = p < nb ? 0 : (p < na ? 1 : 2), cq = q < nb ? 0 : (q < na ? 1 : 2);
    const double fa = Fa_mo[idx], fb = Fb_mo[idx];
    double f = 0.5 * (fa + fb);
    if (cp + cq == 1) f = fb;                       // closed-open
    else if (cp + cq == 3) f = fa;                  // open-virtual
    Fb_mo[idx] = cp != cq ? f : 0.0;
    if (p == q) f += cp == 2 ? shift : (cp == 1 ? 0.5 * shift : 0.0);
    Fa_mo[idx] = f;
}

// out[r] = V[(r + shift) mod m] for the m rows of m entries: row `shift` of V becomes the first row of out
__global__ void rotate_rows_kernel(const double* __restrict__ V, int m, int shift, double* __restrict__ out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)m * m) return;
    const int r = (int)(idx / m), c = (int)(idx % m);
    out[idx] = V[(long long)((r + shift) % m) * m + c];
}

// Unrestricted (two orbital sets) or restricted open-shell (one set: the beta orbitals are the first nb
// alpha orbitals) Hartree-Fock on the density-fitted builds.
class UhfRun {
  public:
    UhfRun(df_handle* h, const df_options* o, int na, int nb, df_result* r, bool restricted = false, double shift = 0.0)
        : h_(h), o_(*o), r_(r), na_(na), nb_(nb), ro_(restricted), shift_(shift) {}
    ~UhfRun() { release(); }

    int run() {
        const auto t_start = std::chrono::steady_clock::now();
        *r_ = df_result{};
        r_->e_nuc = h_->e_nuc;
        if (!h_->built) {
            const auto t0 = std::chrono::steady_clock::now();
            build_B(h_, o_.screen_tau, false, o_.precision == DF_PREC_FP64 ? DF_WHITEN_FP64 : DF_WHITEN_SPLIT);
            r_->t_build_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        }
        n_ = h_->n;
        nn_ = (long long)n_ * n_;
        s_ = h_->stream;
        slices_ = o_.slices;
        const int dsize = std::max(2, std::min(o_.diis_size, DIIS_MAX));
        DF_CUDA(cudaMalloc((void**)&info_, sizeof(int)));
        DF_CUDA(cudaHostAlloc((void**)&pin_, sizeof(double) * 8, cudaHostAllocDefault));
        h_->work1.alloc(nn_);
        h_->work2.alloc(nn_);
        h_->work3.alloc(nn_);
        h_->eps.alloc(2 * (size_t)n_);
        // canonical orthogonaliser X = U s^{-1/2} (eigenvalues of S below 1e-7 dropped)
        DF_CUDA(cudaMemcpyAsync(h_->work1.p, h_->S.p, nn_ * sizeof(double), cudaMemcpyDeviceToDevice, s_));
        eig(h_->work1.p, n_, h_->eps.p);
        std::vector<double> sv(n_);
        int hinfo = 0;
        DF_CUDA(cudaMemcpyAsync(sv.data(), h_->eps.p, n_ * sizeof(double), cudaMemcpyDeviceToHost, s_));
        DF_CUDA(cudaMemcpyAsync(&hinfo, info_, sizeof(int), cudaMemcpyDeviceToHost, s_));
        DF_CUDA(cudaStreamSynchronize(s_));
        if (hinfo != 0) throw Error{DF_E_NUMERIC, "dsyevd of S failed, info " + std::to_string(hinfo)};
        int first = 0;
        while (first < n_ && sv[first] <= 1e-7) ++first;
        nX_ = n_ - first;
        if (nX_ < na_) throw Error{DF_E_NUMERIC, "orthogonal basis smaller than the alpha occupied space"};
        r_->n_dropped = first;
        h_->X.alloc((size_t)n_ * nX_);
        build_x_kernel<<<nblk((long long)n_ * nX_), 256, 0, s_>>>(h_->work1.p, h_->eps.p, n_, first, nX_, h_->X.p);
        DF_CHECK_LAUNCH();
        const long long no = (long long)nX_ * nX_;
        const long long vlen = ro_ ? no : 2 * no;   // DIIS vector: both spins' matrices, or the effective one
        ensure_jk_buffers(h_, std::max(na_, 1));
        auto dalloc = [](double** p, long long count) { DF_CUDA(cudaMalloc((void**)p, sizeof(double) * count)); };
        dalloc(&D_, 3 * nn_);               // D_a | D_b | D_a + D_b
        dalloc(&F_, 2 * nn_);               // F_a | F_b
        dalloc(&Kb_, nn_);
        dalloc(&C_, (long long)n_ * (na_ + std::max(nb_, 1)));   // C_a (n x na) | C_b (n x nb)
        dalloc(&Fo_, 2 * no);               // F'_a | F'_b
        dalloc(&V_, 2 * no);                // eigenvectors (rows) of the alpha and beta Roothaan steps
        dalloc(&T1_, (long long)n_ * nX_);
        dalloc(&diisF_, DIIS_MAX * 2 * no);
        dalloc(&diisE_, DIIS_MAX * 2 * no);
        dalloc(&Bm_, DIIS_MAX * DIIS_MAX + 8 + DIIS_MAX);   // B matrix | scalars | coefficients
        DF_CUDA(cudaMalloc((void**)&ints_, sizeof(int) * (2 * DIIS_MAX + 4)));
        DF_CUDA(cudaMemsetAsync(ints_, 0, sizeof(int) * (2 * DIIS_MAX + 4), s_));
        double* scal = Bm_ + DIIS_MAX * DIIS_MAX;
        double* coef = scal + 8;
        int* slotp = ints_ + 2 * DIIS_MAX + 3;
        std::vector<int> present(DIIS_MAX, 0), order;
        std::vector<int> ctl(2 * DIIS_MAX + 4, 0);
        if (o_.guess == DF_GUESS_SPIN) {
            // natural orbitals of the last run's spin densities: for each spin the eigenvectors of
            // X^T S D_s S X, the n_s of largest occupation first
            if (!h_->Dspin.p) throw Error{DF_E_STATE, "scf_run_uhf: no spin densities of an earlier open-shell run"};
            for (int sp = 0; sp < 2; ++sp) {
                const int nocc = sp == 0 ? na_ : nb_;
                dgemm(s_, false, false, n_, n_, n_, 1.0, h_->S.p, n_, h_->Dspin.p + sp * nn_, n_, 0.0, h_->work1.p, n_);
                dgemm(s_, false, false, n_, n_, n_, 1.0, h_->work1.p, n_, h_->S.p, n_, 0.0, h_->work2.p, n_);
                to_orth(h_->work2.p, Fo_ + sp * no);
                eig(Fo_ + sp * no, nX_, h_->eps.p + sp * n_);   // ascending: the occupied are the last rows
                rotate_rows_kernel<<<nblk(no), 256, 0, s_>>>(Fo_ + sp * no, nX_, nX_ - nocc, V_ + sp * no);
                DF_CHECK_LAUNCH();
                double* C = C_ + (sp == 0 ? 0 : (long long)n_ * na_);
                double* D = D_ + sp * nn_;
                if (nocc > 0) {
                    dgemm(s_, false, true, n_, nocc, nX_, 1.0, h_->X.p, nX_, V_ + sp * no, nX_, 0.0, C, nocc);
                    dgemm(s_, false, true, n_, n_, nocc, 1.0, C, nocc, C, nocc, 0.0, D, n_);
                } else {
                    DF_CUDA(cudaMemsetAsync(D, 0, sizeof(double) * nn_, s_));
                }
            }
            add_kernel2<<<nblk(nn_), 256, 0, s_>>>(D_, D_ + nn_, nn_, D_ + 2 * nn_);
            DF_CHECK_LAUNCH();
        } else {
            // core-Hamiltonian start for both spins
            to_orth(h_->H.p, Fo_);
            DF_CUDA(cudaMemcpyAsync(Fo_ + no, Fo_, sizeof(double) * no, cudaMemcpyDeviceToDevice, s_));
            roothaan(Fo_);
        }
        const auto t_iter = std::chrono::steady_clock::now();
        double e_old = 0.0, jk_ms = 0.0;
        int status = DF_E_NOTCONV;
        cudaEvent_t j0, j1;
        DF_CUDA(cudaEventCreate(&j0));
        DF_CUDA(cudaEventCreate(&j1));
        h_->history.clear();
        for (int it = 1; it <= o_.max_iter; ++it) {
            DF_CUDA(cudaEventRecord(j0, s_));
            coulomb_fp64(h_, D_ + 2 * nn_, h_->dJ.p);
            exchange_only(h_, C_, na_, o_.precision, slices_, h_->dK.p);
            if (nb_ > 0) exchange_only(h_, C_ + (long long)n_ * na_, nb_, o_.precision, slices_, Kb_);
            else DF_CUDA(cudaMemsetAsync(Kb_, 0, sizeof(double) * nn_, s_));
            DF_CUDA(cudaEventRecord(j1, s_));
            fock_kernel<<<nblk(nn_), 256, 0, s_>>>(h_->H.p, h_->dJ.p, h_->dK.p, nn_, F_);
            DF_CHECK_LAUNCH();
            fock_kernel<<<nblk(nn_), 256, 0, s_>>>(h_->H.p, h_->dJ.p, Kb_, nn_, F_ + nn_);
            DF_CHECK_LAUNCH();
            energy_kernel<<<1, 1024, 0, s_>>>(D_, h_->H.p, h_->dJ.p, h_->dK.p, nn_, scal);
            DF_CHECK_LAUNCH();
            energy_kernel<<<1, 1024, 0, s_>>>(D_ + nn_, h_->H.p, h_->dJ.p, Kb_, nn_, scal + 4);
            DF_CHECK_LAUNCH();
            // DIIS slot of this iteration
            int slot = 0;
            if ((int)order.size() < dsize) {
                while (present[slot]) ++slot;
            } else {
                slot = order.front();
                order.erase(order.begin());
                present[slot] = 0;
            }
            double* E = diisE_ + (long long)slot * 2 * no;
            if (ro_) {
                // F_s in the orbital basis (V: current orbitals as rows), the effective matrix and its error,
                // both taken back to the orthogonal basis: F'_eff = V^T F_eff,mo V
                for (int sp = 0; sp < 2; ++sp) {
                    to_orth(F_ + sp * nn_, Fo_ + sp * no);
                    dgemm(s_, false, false, nX_, nX_, nX_, 1.0, V_, nX_, Fo_ + sp * no, nX_, 0.0, h_->work1.p, nX_);
                    dgemm(s_, false, true, nX_, nX_, nX_, 1.0, h_->work1.p, nX_, V_, nX_, 0.0,
                          sp == 0 ? h_->work2.p : h_->work3.p, nX_);
                }
                rohf_effective_kernel<<<nblk(no), 256, 0, s_>>>(h_->work2.p, h_->work3.p, nX_, na_, nb_, shift_);
                DF_CHECK_LAUNCH();
                dgemm(s_, true, false, nX_, nX_, nX_, 1.0, V_, nX_, h_->work2.p, nX_, 0.0, h_->work1.p, nX_);
                dgemm(s_, false, false, nX_, nX_, nX_, 1.0, h_->work1.p, nX_, V_, nX_, 0.0, Fo_, nX_);
                dgemm(s_, true, false, nX_, nX_, nX_, 1.0, V_, nX_, h_->work3.p, nX_, 0.0, h_->work1.p, nX_);
                dgemm(s_, false, false, nX_, nX_, nX_, 1.0, h_->work1.p, nX_, V_, nX_, 0.0, E, nX_);
            }
            for (int sp = 0; sp < 2 && !ro_; ++sp) {
                const int nocc = sp == 0 ? na_ : nb_;
                double* Fos = Fo_ + sp * no;
                to_orth(F_ + sp * nn_, Fos);
                if (nocc > 0) {
                    const double* Vo = V_ + sp * no;   // occupied rows first
                    dgemm(s_, false, true, nX_, nocc, nX_, 1.0, Fos, nX_, Vo, nX_, 0.0, h_->work2.p, nocc);
                    dgemm(s_, false, false, nX_, nX_, nocc, 1.0, h_->work2.p, nocc, Vo, nX_, 0.0, h_->work1.p, nX_);
                    antisym_kernel<<<nblk(no), 256, 0, s_>>>(h_->work1.p, nX_, 1.0, E + sp * no);
                    DF_CHECK_LAUNCH();
                } else {
                    DF_CUDA(cudaMemsetAsync(E + sp * no, 0, sizeof(double) * no, s_));
                }
            }
            absmax_kernel<<<1, 1024, 0, s_>>>(E, vlen, scal + 3);
            DF_CHECK_LAUNCH();
            DF_CUDA(cudaMemcpyAsync(pin_, scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s_));
            DF_CUDA(cudaStreamSynchronize(s_));
            const double this_jk = elapsed_ms(j0, j1);
            jk_ms += this_jk;
            const double energy = pin_[0] + 0.5 * pin_[1] - 0.5 * pin_[2] + pin_[4] + 0.5 * pin_[5] - 0.5 * pin_[6] +
                                  h_->e_nuc;
            const double err = pin_[3];
            h_->history.insert(h_->history.end(), {(double)it, energy, it > 1 ? energy - e_old : 0.0, err,
                                                   o_.precision == DF_PREC_SPLIT ? (double)slices_ : 0.0, this_jk});
            r_->iterations = it;
            r_->energy = energy;
            r_->e_one = pin_[0] + pin_[4];
            r_->e_coul = 0.5 * (pin_[1] + pin_[5]);
            r_->e_exch = -0.5 * (pin_[2] + pin_[6]);
            r_->last_err = err;
            r_->last_dE = it > 1 ? energy - e_old : 0.0;
            if (!std::isfinite(energy) || !std::isfinite(err)) {
                status = DF_E_NUMERIC;
                break;
            }
            const bool late_ready = o_.precision != DF_PREC_SPLIT || slices_ >= SPLIT_LATE_SLICES;
            if (it > 1 && late_ready && std::fabs(energy - e_old) < o_.conv_E && err < o_.conv_err) {
                status = DF_OK;
                break;
            }
            e_old = energy;
            if (o_.precision == DF_PREC_SPLIT && slices_ < SPLIT_LATE_SLICES && err < SPLIT_RAMP_ERR) {
                slices_ = SPLIT_LATE_SLICES;   // the DIIS subspace restarts with the finer exchange
                r_->ramp_iteration = it + 1;
                for (int q : order) present[q] = 0;
                order.clear();
            }
            DF_CUDA(cudaMemcpyAsync(diisF_ + (long long)slot * 2 * no, Fo_, sizeof(double) * vlen,
                                    cudaMemcpyDeviceToDevice, s_));
            present[slot] = 1;
            order.push_back(slot);
            for (int q = 0; q < DIIS_MAX; ++q) ctl[q] = present[q];
            for (size_t q = 0; q < order.size(); ++q) ctl[DIIS_MAX + q] = order[q];
            ctl[2 * DIIS_MAX + 3] = slot;
            DF_CUDA(cudaMemcpyAsync(ints_, ctl.data(), sizeof(int) * (2 * DIIS_MAX + 4), cudaMemcpyHostToDevice, s_));
            diis_dots_kernel<<<DIIS_MAX, 256, 0, s_>>>(diisE_, 2 * no, vlen, slotp, ints_, DIIS_MAX, Bm_);
            DF_CHECK_LAUNCH();
            if (it >= 2 && order.size() >= 2) {
                diis_solve_kernel<<<1, 1, 0, s_>>>(Bm_, ints_ + DIIS_MAX, (int)order.size(), coef, ints_ + 2 * DIIS_MAX);
                DF_CHECK_LAUNCH();
                diis_combine_kernel<<<nblk(vlen), 256, 0, s_>>>(diisF_, 2 * no, vlen, ints_ + DIIS_MAX,
                                                                 (int)order.size(), coef, Fo_);
                DF_CHECK_LAUNCH();
                int singular = 0;
                DF_CUDA(cudaMemcpyAsync(&singular, ints_ + 2 * DIIS_MAX, sizeof(int), cudaMemcpyDeviceToHost, s_));
                DF_CUDA(cudaStreamSynchronize(s_));   // ctl (host) is rewritten next iteration
                if (singular && order.size() > 1) {   // drop the oldest vector from the subspace
                    present[order.front()] = 0;
                    order.erase(order.begin());
                }
            } else {
                DF_CUDA(cudaStreamSynchronize(s_));   // ctl (host) is rewritten next iteration
            }
            roothaan(Fo_);
        }
        cudaEventDestroy(j0);
        cudaEventDestroy(j1);
        r_->s2 = spin_s2();
        r_->converged = status == DF_OK;
        r_->status = status;
        r_->t_iter_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_iter).count();
        r_->t_jk_s = jk_ms / 1000.0;
        r_->t_total_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        // the total density becomes the handle's D (df_get_matrix), the spin densities its spin buffers
        if (!h_->Dm.p) h_->Dm.alloc(nn_);
        h_->Dspin.alloc(2 * nn_);
        DF_CUDA(cudaMemcpyAsync(h_->Dm.p, D_ + 2 * nn_, sizeof(double) * nn_, cudaMemcpyDeviceToDevice, s_));
        DF_CUDA(cudaMemcpyAsync(h_->Dspin.p, D_, sizeof(double) * 2 * nn_, cudaMemcpyDeviceToDevice, s_));
        DF_CUDA(cudaStreamSynchronize(s_));
        return status;
    }

  private:
    // Roothaan step for both spins from F'_a | F'_b held in Fs (overwritten by the eigenvectors)
    void roothaan(double* Fs) {
        const long long no = (long long)nX_ * nX_;
        for (int sp = 0; sp < 2; ++sp) {
            const int nocc = sp == 0 ? na_ : nb_;
            if (ro_ && sp == 1) {
                // one orbital set: the beta determinant takes the first nb orbitals of the alpha step
                DF_CUDA(cudaMemcpyAsync(V_ + no, V_, sizeof(double) * no, cudaMemcpyDeviceToDevice, s_));
                DF_CUDA(cudaMemcpyAsync(h_->eps.p + n_, h_->eps.p, sizeof(double) * nX_, cudaMemcpyDeviceToDevice, s_));
            } else {
                DF_CUDA(cudaMemcpyAsync(V_ + sp * no, Fs + sp * no, sizeof(double) * no, cudaMemcpyDeviceToDevice, s_));
                eig(V_ + sp * no, nX_, h_->eps.p + sp * n_);
            }
            double* C = C_ + (sp == 0 ? 0 : (long long)n_ * na_);
            double* D = D_ + sp * nn_;
            if (nocc > 0) {
                dgemm(s_, false, true, n_, nocc, nX_, 1.0, h_->X.p, nX_, V_ + sp * no, nX_, 0.0, C, nocc);
                dgemm(s_, false, true, n_, n_, nocc, 1.0, C, nocc, C, nocc, 0.0, D, n_);
            } else {
                DF_CUDA(cudaMemsetAsync(D, 0, sizeof(double) * nn_, s_));
            }
        }
        add_kernel2<<<nblk(nn_), 256, 0, s_>>>(D_, D_ + nn_, nn_, D_ + 2 * nn_);
        DF_CHECK_LAUNCH();
    }

    // <S^2> = S_z (S_z + 1) + n_beta - tr(D_a S D_b S)
    double spin_s2() {
        dgemm(s_, false, false, n_, n_, n_, 1.0, D_, n_, h_->S.p, n_, 0.0, h_->work1.p, n_);          // D_a S
        dgemm(s_, false, false, n_, n_, n_, 1.0, D_ + nn_, n_, h_->S.p, n_, 0.0, h_->work2.p, n_);    // D_b S
        transpose_kernel<<<nblk(nn_), 256, 0, s_>>>(h_->work2.p, n_, h_->work3.p);
        double* scal = Bm_ + DIIS_MAX * DIIS_MAX;
        energy_kernel<<<1, 1024, 0, s_>>>(h_->work1.p, h_->work3.p, h_->work3.p, h_->work3.p, nn_, scal);
        DF_CHECK_LAUNCH();
        double tr = 0.0;
        DF_CUDA(cudaMemcpyAsync(&tr, scal, sizeof(double), cudaMemcpyDeviceToHost, s_));
        DF_CUDA(cudaStreamSynchronize(s_));
        const double sz = 0.5 * (na_ - nb_);
        return sz * (sz + 1.0) + nb_ - tr;
    }

    void eig(double* A, int m, double* w) {
        int lw = 0;
        DF_SOLVER(cusolverDnDsyevd_bufferSize(h_->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, m, A, m, w, &lw));
        if (lw > lwork_) {
            if (work_) cudaFree(work_);
            work_ = nullptr;
            DF_CUDA(cudaMalloc((void**)&work_, sizeof(double) * lw));
            lwork_ = lw;
        }
        DF_SOLVER(cusolverDnDsyevd(h_->solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, m, A, m, w, work_,
                                   lwork_, info_));
    }

    // Fo = X^T Fm X (nX x nX)
    void to_orth(const double* Fm, double* Fo) {
        dgemm(s_, false, false, n_, nX_, n_, 1.0, Fm, n_, h_->X.p, nX_, 0.0, T1_, nX_);
        dgemm(s_, true, false, nX_, nX_, n_, 1.0, h_->X.p, nX_, T1_, nX_, 0.0, Fo, nX_);
    }

    void release() {
        if (s_) cudaStreamSynchronize(s_);
        double* bufs[] = {D_, F_, Kb_, C_, Fo_, V_, T1_, diisF_, diisE_, Bm_, work_};
        for (double* b : bufs)
            if (b) cudaFree(b);
        if (ints_) cudaFree(ints_);
        if (info_) cudaFree(info_);
        if (pin_) cudaFreeHost(pin_);
        D_ = F_ = Kb_ = C_ = Fo_ = V_ = T1_ = diisF_ = diisE_ = Bm_ = work_ = nullptr;
        ints_ = info_ = nullptr;
        pin_ = nullptr;
    }

    df_handle* h_;
    df_options o_;
    df_result* r_;
    int na_, nb_;
    bool ro_;
    double shift_;
    int n_ = 0, nX_ = 0, slices_ = 3, lwork_ = 0;
    long long nn_ = 0;
    cudaStream_t s_ = nullptr;
    double *D_ = nullptr, *F_ = nullptr, *Kb_ = nullptr, *C_ = nullptr, *Fo_ = nullptr, *V_ = nullptr, *T1_ = nullptr;
    double *diisF_ = nullptr, *diisE_ = nullptr, *Bm_ = nullptr, *work_ = nullptr, *pin_ = nullptr;
    int *ints_ = nullptr, *info_ = nullptr;
};

}  // namespace

// Fractional-occupation SCF of one atom (handle ha, nelec electrons), FP64, converged to |dE| < 1e-11 and
// max|e| < 1e-9: Cw (host, n x m row-major) receives the weighted occupied orbitals of the converged
// density, D = 2 Cw Cw^T.
void atomic_scf(df_handle* ha, double nelec, std::vector<double>& Cw, int& m) {
    df_options o{};
    o.conv_E = 1e-11;
    o.conv_err = 1e-9;
    o.max_iter = 200;
    o.diis_size = 8;
    o.guess = DF_GUESS_CORE;
    o.precision = DF_PREC_FP64;
    o.slices = 3;
    df_result r{};
    ScfRun run(ha, &o, &r);
    run.set_fractional(nelec);
    run.begin();
    while (!run.done()) {
        run.enqueue_iteration();
        run.finish_iteration();
    }
    if (run.status() != DF_OK)
        throw Error{DF_E_NUMERIC, "superposition-of-atomic-densities guess: the SCF of an atom (" +
                                      std::to_string(nelec) + " electrons) did not converge"};
    m = run.occupied_count();
    Cw.resize((size_t)ha->n * m);
    DF_CUDA(cudaStreamSynchronize(ha->stream));
    DF_CUDA(cudaMemcpy(Cw.data(), run.occupied_factor(), sizeof(double) * Cw.size(), cudaMemcpyDeviceToHost));
}

int scf_drive_uhf(df_handle* h, const df_options* o, int nalpha, int nbeta, df_result* r) {
    UhfRun run(h, o, nalpha, nbeta, r);
    return run.run();
}

int scf_drive_rohf(df_handle* h, const df_options* o, int nalpha, int nbeta, double level_shift, df_result* r) {
    UhfRun run(h, o, nalpha, nbeta, r, true, level_shift);
    return run.run();
}

int scf_drive(df_handle* h, const df_options* o, df_result* r, const double* guess) {
    ScfRun run(h, o, r, guess);
    DevBuf<double> C0;
    if (!guess && o->guess == DF_GUESS_SAD) {
        int m0 = 0;
        sad_factor(h, C0, m0);
        run.set_initial_factor(C0.p, m0);
    }
    run.begin();
    while (!run.done()) {
        run.enqueue_iteration();
        run.finish_iteration();
    }
    return run.status();
}

// Many molecules on one host thread, driven by completion events: a molecule whose enqueued iteration
// has finished on its stream is advanced (convergence test, DIIS, Roothaan step, next iteration) without
// waiting for the others, and one more molecule is started per pass, so its B build (which waits only
// on its own stream) runs while the queued iterations of the others proceed on the GPU.
int scf_drive_batch(df_handle** hs, int nmol, const df_options* o, df_result* rs) {
    std::vector<std::unique_ptr<ScfRun>> runs;
    std::vector<DevBuf<double>> factors(nmol);   // SAD starting factors, alive until the runs end
    for (int i = 0; i < nmol; ++i) {
        hs[i]->sync_timing = false;
        runs.emplace_back(new ScfRun(hs[i], o, &rs[i]));
    }
    int status = DF_OK;
    try {
        // the three-centre integrals of every molecule without B in one grouped launch per class; each
        // molecule's metric factor and whitening follow when the driver starts it
        build_B_batch(hs, nmol, o->screen_tau, false, o->precision == DF_PREC_FP64 ? DF_WHITEN_FP64 : DF_WHITEN_SPLIT,
                      false);
        if (o->guess == DF_GUESS_SAD)
            for (int i = 0; i < nmol; ++i) {
                int m0 = 0;
                sad_factor(hs[i], factors[i], m0);
                runs[i]->set_initial_factor(factors[i].p, m0);
            }
        // DFHF_BATCH_TRACE=1: host time per part of the loop, printed to stderr at the end
        const char* tv = std::getenv("DFHF_BATCH_TRACE");
        const bool trace = tv && tv[0] == '1';
        double t_begin = 0, t_finish = 0, t_enqueue = 0, t_idle = 0;
        long long n_iter = 0;
        using tclk = std::chrono::steady_clock;
        auto since = [](tclk::time_point a) { return std::chrono::duration<double>(tclk::now() - a).count(); };
        const auto t_all = tclk::now();
        int started = 0, finished = 0;
        while (finished < nmol) {
            bool progressed = false;
            for (int i = 0; i < started; ++i) {
                ScfRun& r = *runs[i];
                if (r.done() || !r.ready()) continue;
                auto t0 = tclk::now();
                r.finish_iteration();
                t_finish += since(t0);
                ++n_iter;
                if (r.done()) {
                    ++finished;
                } else {
                    t0 = tclk::now();
                    r.enqueue_iteration();
                    t_enqueue += since(t0);
                }
                progressed = true;
            }
            if (started < nmol) {
                auto t0 = tclk::now();
                runs[started]->begin();
                t_begin += since(t0);
                t0 = tclk::now();
                runs[started]->enqueue_iteration();
                t_enqueue += since(t0);
                ++started;
                progressed = true;
            }
            if (!progressed) {
                const auto t0 = tclk::now();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                t_idle += since(t0);
            }
        }
        if (trace)
            std::fprintf(stderr,
                         "batch trace: %d molecules, %lld iterations, %.3f s: begin (B build, orthogonaliser) %.3f s, "
                         "finish %.3f s, enqueue %.3f s, waiting %.3f s\n",
                         nmol, n_iter, since(t_all), t_begin, t_finish, t_enqueue, t_idle);
        for (auto& r : runs)
            if (r->status() != DF_OK && status == DF_OK) status = r->status();
    } catch (...) {
        for (int i = 0; i < nmol; ++i) hs[i]->sync_timing = true;
        throw;
    }
    for (int i = 0; i < nmol; ++i) hs[i]->sync_timing = true;
    return status;
}

}  // namespace dfhf
