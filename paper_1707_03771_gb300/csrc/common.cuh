// Shared definitions of the CUDA library: error handling, shell tables and the handle.
#pragma once
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/dfhf.h"

namespace dfhf {

// ------------------------------------------------------------------------------------------------
// errors: every internal failure becomes a status code plus a message stored on the handle
// ------------------------------------------------------------------------------------------------
struct Error {
    int code;
    std::string msg;
};

#define DF_CUDA(call)                                                                            \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            throw ::dfhf::Error{e_ == cudaErrorMemoryAllocation ? DF_E_NOMEM : DF_E_CUDA,        \
                                std::string(#call) + ": " + cudaGetErrorString(e_)};             \
    } while (0)

#define DF_SOLVER(call)                                                                          \
    do {                                                                                         \
        cusolverStatus_t s_ = (call);                                                            \
        if (s_ != CUSOLVER_STATUS_SUCCESS)                                                       \
            throw ::dfhf::Error{DF_E_CUDA, std::string(#call) + ": cusolver status " +            \
                                               std::to_string((int)s_)};                         \
    } while (0)

#define DF_CHECK_LAUNCH() DF_CUDA(cudaGetLastError())

// ------------------------------------------------------------------------------------------------
// shells on the device (structure of arrays)
// ------------------------------------------------------------------------------------------------
struct ShellTable {
    int count = 0;
    int* l = nullptr;           // angular momentum
    int* off = nullptr;         // first function index
    double* alpha = nullptr;    // exponent
    double* norm = nullptr;     // normalisation of the real solid harmonic Gaussian
    double* xyz = nullptr;      // centre, 3 per shell
};

// shell pairs / triples of one angular-momentum class: entries are shell indices
struct ClassList {
    int la = 0, lb = 0;         // la >= lb (pairs) ; for aux lists lb unused
    int count = 0;
    int2* d_pairs = nullptr;    // (a, b) with l(a) = la, l(b) = lb
};

// packed layout of one auxiliary row of B: tiles of TS x TS over (I >= J) tile pairs
constexpr int TS = 64;

struct Packing {
    int n = 0, np = 0, nt = 0;  // functions, padded functions, tiles per dimension
    long long ntp = 0;          // tile pairs I >= J
    long long row = 0;          // doubles per auxiliary row = ntp * TS * TS
};

__host__ __device__ inline long long tile_pair(int I, int J) { return (long long)I * (I + 1) / 2 + J; }

// position of element (mu, nu) in a packed row; for mu, nu in the same tile the mirror is stored too
__host__ __device__ inline long long packed_index(int mu, int nu) {
    int I = mu / TS, J = nu / TS;
    if (I >= J) return tile_pair(I, J) * TS * TS + (mu % TS) * TS + (nu % TS);
    return tile_pair(J, I) * TS * TS + (nu % TS) * TS + (mu % TS);
}

// ------------------------------------------------------------------------------------------------
// the handle
// ------------------------------------------------------------------------------------------------
template <class T>
struct DevBuf {
    // owns one device allocation: move-only, released by its owner's scope (or earlier by release())
    T* p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) {
        o.p = nullptr;
        o.n = 0;
    }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            n = o.n;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count) {
        release();
        if (count == 0) return;
        DF_CUDA(cudaMalloc((void**)&p, count * sizeof(T)));
        n = count;
    }
    void zero(cudaStream_t s) {
        if (p) DF_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

struct SplitState;   // split-precision work buffers (split_k.cu)

}  // namespace dfhf

struct df_handle {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    cusolverDnHandle_t solver = nullptr;
    std::string last_error;

    // system
    std::vector<df_atom> atoms;
    std::vector<df_shell> basis, aux;
    int n = 0, naux = 0, nocc = 0, nelec = 0;
    double e_nuc = 0.0;
    dfhf::Packing pk;

    // device tables
    dfhf::ShellTable dbas, daux;
    dfhf::DevBuf<double> d_atom_xyz, d_atom_Z;
    std::vector<dfhf::ClassList> pair_classes;     // orbital shell pairs by (la >= lb)
    std::vector<dfhf::ClassList> aux_pairs;        // auxiliary shell pairs P >= Q by (lP >= lQ)
    std::vector<std::vector<int>> aux_by_l;         // auxiliary shells by l (host)
    dfhf::DevBuf<int> d_aux_by_l[DF_LMAX_AUX + 1];

    // one-electron and metric
    dfhf::DevBuf<double> S, T, V, H, metric, Linv;

    // three-index tensors, packed rows of length pk.row
    dfhf::DevBuf<double> A3c, B;
    bool built = false;
    int whitening = DF_WHITEN_SPLIT;   // how B was whitened (DF_WHITEN_*)
    bool a3c_ready = false;            // A3c already holds (P|mu nu) (grouped integrals of a batch)

    // J/K work
    dfhf::DevBuf<double> Dw, gamma, Jp, Y, Kpart, Cpad, dD, dC, dJ, dK;
    dfhf::DevBuf<int2> ktiles;
    int nocc_alloc = 0;
    dfhf::SplitState* split = nullptr;

    // SCF state
    dfhf::DevBuf<double> X, F, Fx, Dm, C, eps, work1, work2, work3, diisF, diisE, diisB;
    dfhf::DevBuf<double> Dspin;   // alpha | beta densities of the last UHF run
    int nX = 0;
    int ndrop = 0;

    double timings_ms[20] = {0};
    int exchange_launches = 0;     // kernel launches of the last exchange build
    std::vector<double> history;   // per SCF iteration: iteration, energy, dE, max|e|, slices, J/K ms
    bool sync_timing = true;       // per-kernel event timings (the batch driver turns them off)
    int* tc_err_host = nullptr;    // set by the SCF driver: the tensor-core kernels' timeout flag is copied
                                   // here (pinned) instead of being read back with a synchronisation
    double* noalloc_scratch = nullptr;   // device address of the library's static Coulomb scratch array on
                                         // this handle's device, resolved by df_init (null if that failed)
    std::string noalloc_error;           // why it could not be resolved
};

namespace dfhf {
// handle creation (capi.cu); closed_shell = false admits any electron count (atoms of the SAD guess)
int init_handle(const df_atom* atoms, int natom, const df_shell* basis, int nbasis_sh, const df_shell* aux,
                int naux_sh, int charge, df_handle** out, bool closed_shell);

// integral builders (integrals.cu)
void compute_one_electron(df_handle* h);
void compute_metric(df_handle* h);
void compute_three_center(df_handle* h, double* out, double tau);
void compute_three_center_grouped(const std::vector<df_handle*>& hs, const std::vector<double*>& outs,
                                  cudaStream_t s);
void build_B(df_handle* h, double tau, bool keep, int whitening);
void build_B_batch(df_handle** hs, int n, double tau, bool keep, int whitening, bool whiten_now);
void rys_eval(const double* dT, int count, int n, double* dx, double* dw, cudaStream_t s);

// FP64 dense kernels (dense.cu)
// C = alpha * op(A) * op(B) + beta * C, row-major, op(X) = X or X^T
void dgemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
           const double* B, int ldb, double beta, double* C, int ldc);
// C = alpha * Linv * A for lower-triangular Linv (m x m), A (m x ncol), lda = ldc = row stride
void dtrmm_lower(cudaStream_t s, int m, long long ncol, const double* Linv, const double* A, double* C,
                 long long ld);

// J/K (jk.cu)
void jk_fp64(df_handle* h, const double* dD, const double* dC, int nocc, double* dJ, double* dK);
void ensure_jk_buffers(df_handle* h, int nocc);
void coulomb_fp64(df_handle* h, const double* dD, double* dJ);
void pad_occupied(df_handle* h, const double* dC, int nocc, int ldy);
// Y_{P,mu i} = sum_nu B_{P,mu nu} C_{nu i} from the packed FP64 B (Y: naux x np x ldy)
void y_transform_fp64(cudaStream_t s, const double* B, long long row, int nt, int naux, const double* Cp, int ldy,
                      int ncol, double* Y);
void exchange_fp64(df_handle* h, int nocc, double* dK);
int k_splits(const df_handle* h);
void unpack_rows(df_handle* h, const double* packed, int p0, int count, double* dout);

// split precision (split_k.cu)
void exchange_split(df_handle* h, const double* dC, int nocc, int slices, double* dK);
void split_clear_error(df_handle* h);
// the split exchange's Y buffer viewed as doubles, if it holds at least `elems` of them (else nullptr)
double* split_y_buffer(df_handle* h, long long elems);
void free_split(df_handle* h);

// static scratch of df_coulomb_noalloc (coulomb_noalloc.cu): device address of the array on the current
// device; loads the library's module holding it if the runtime has not loaded it yet
int noalloc_scratch_address(double** out, std::string* why);

// SCF (scf.cu)
int scf_drive(df_handle* h, const df_options* o, df_result* r, const double* guess = nullptr);
void atomic_scf(df_handle* ha, double nelec, std::vector<double>& Cw, int& m);
std::vector<double> aufbau_occupations(const std::vector<double>& eps, double nelec);

// superposition of atomic densities (sad.cu): C0 (device, n x m0) with D0 = 2 C0 C0^T
void sad_factor(df_handle* h, DevBuf<double>& C0, int& m0);
int scf_drive_batch(df_handle** hs, int nmol, const df_options* o, df_result* rs);
int scf_drive_uhf(df_handle* h, const df_options* o, int nalpha, int nbeta, df_result* r);
int scf_drive_rohf(df_handle* h, const df_options* o, int nalpha, int nbeta, double level_shift, df_result* r);

double elapsed_ms(cudaEvent_t a, cudaEvent_t b);

// CUDA events marking the phases of one build for the per-phase timings; none at all when `on` is false
// (batched runs, and stream capture, where a call's own events cannot be recorded and then destroyed)
struct PhaseTimer {
    static constexpr int MAXEV = 8;
    cudaEvent_t ev[MAXEV] = {};
    int count = 0;
    bool on = false;
    PhaseTimer(bool enabled, int n) : count(n < MAXEV ? n : MAXEV), on(enabled) {
        if (on)
            for (int i = 0; i < count; ++i) DF_CUDA(cudaEventCreate(&ev[i]));
    }
    PhaseTimer(const PhaseTimer&) = delete;
    PhaseTimer& operator=(const PhaseTimer&) = delete;
    void mark(int i, cudaStream_t s) {
        if (on) DF_CUDA(cudaEventRecord(ev[i], s));
    }
    double ms(int a, int b) const { return elapsed_ms(ev[a], ev[b]); }
    void sync(int i) {
        if (on) DF_CUDA(cudaEventSynchronize(ev[i]));
    }
    ~PhaseTimer() {
        if (on)
            for (int i = 0; i < count; ++i) cudaEventDestroy(ev[i]);
    }
};
}  // namespace dfhf
