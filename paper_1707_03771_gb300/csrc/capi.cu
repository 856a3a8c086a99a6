// The C ABI (include/dfhf.h): handle set-up, shell tables, B construction and the public entry
// points. Every entry point converts internal exceptions into status codes.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>

#include <cstdlib>
#include <string>

#include "common.cuh"
#include "ozaki.cuh"

namespace dfhf {

void rys_eval(const double* dT, int count, int n, double* dx, double* dw, cudaStream_t s);
const double* rys_table_host();
void whiten_ozaki(cudaStream_t s, int naux, long long ncol, long long ld, const double* Linv, const double* A,
                  double* B);
void whiten_float_float(cudaStream_t s, int m, long long ncol, const double* Linv, double* Lff, double* A, double* B,
                        long long ld, bool restore_a);
void coulomb_kernels_load();
void whiten_fp64_inplace(cudaStream_t s, int m, long long ncol, const double* L, double* A, long long ld);

namespace {

// normalisation of N S_lm exp(-alpha r^2) with S_lm the real solid harmonics (norm independent of m):
// int S_lm^2 exp(-2 alpha r^2) d^3r = pi^{3/2} (2l-1)!! / (2^l (2 alpha)^{l+3/2})
double shell_norm(int l, double alpha) {
    double dfact = 1.0;
    for (int k = 2 * l - 1; k > 1; k -= 2) dfact *= k;
    const double pi = 3.14159265358979323846;
    const double integral = std::pow(pi, 1.5) * dfact / (std::pow(2.0, l) * std::pow(2.0 * alpha, l + 1.5));
    return 1.0 / std::sqrt(integral);
}

void upload_shells(const std::vector<df_shell>& sh, ShellTable& t, cudaStream_t s) {
    const int n = (int)sh.size();
    std::vector<int> l(n), off(n);
    std::vector<double> a(n), nrm(n), xyz(3 * n);
    int o = 0;
    for (int i = 0; i < n; ++i) {
        l[i] = sh[i].l;
        off[i] = o;
        o += 2 * sh[i].l + 1;
        a[i] = sh[i].exponent;
        nrm[i] = shell_norm(sh[i].l, sh[i].exponent);
        for (int d = 0; d < 3; ++d) xyz[3 * i + d] = sh[i].center[d];
    }
    t.count = n;
    DF_CUDA(cudaMalloc((void**)&t.l, sizeof(int) * n));
    DF_CUDA(cudaMalloc((void**)&t.off, sizeof(int) * n));
    DF_CUDA(cudaMalloc((void**)&t.alpha, sizeof(double) * n));
    DF_CUDA(cudaMalloc((void**)&t.norm, sizeof(double) * n));
    DF_CUDA(cudaMalloc((void**)&t.xyz, sizeof(double) * 3 * n));
    DF_CUDA(cudaMemcpyAsync(t.l, l.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    DF_CUDA(cudaMemcpyAsync(t.off, off.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    DF_CUDA(cudaMemcpyAsync(t.alpha, a.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    DF_CUDA(cudaMemcpyAsync(t.norm, nrm.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    DF_CUDA(cudaMemcpyAsync(t.xyz, xyz.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s));
    DF_CUDA(cudaStreamSynchronize(s));
}

void free_shells(ShellTable& t) {
    cudaFree(t.l);
    cudaFree(t.off);
    cudaFree(t.alpha);
    cudaFree(t.norm);
    cudaFree(t.xyz);
    t = ShellTable{};
}

// shell pairs (M >= N) grouped by class (la >= lb), the higher l first in each pair
std::vector<ClassList> make_pairs(const std::vector<df_shell>& sh, int lmax, cudaStream_t s) {
    std::vector<std::vector<int2>> buckets((lmax + 1) * (lmax + 1));
    for (int M = 0; M < (int)sh.size(); ++M)
        for (int N = 0; N <= M; ++N) {
            int a = M, b = N;
            if (sh[a].l < sh[b].l) std::swap(a, b);
            buckets[sh[a].l * (lmax + 1) + sh[b].l].push_back(make_int2(a, b));
        }
    std::vector<ClassList> out;
    for (int la = 0; la <= lmax; ++la)
        for (int lb = 0; lb <= la; ++lb) {
            auto& v = buckets[la * (lmax + 1) + lb];
            ClassList c;
            c.la = la;
            c.lb = lb;
            c.count = (int)v.size();
            if (c.count) {
                DF_CUDA(cudaMalloc((void**)&c.d_pairs, sizeof(int2) * c.count));
                DF_CUDA(cudaMemcpyAsync(c.d_pairs, v.data(), sizeof(int2) * c.count, cudaMemcpyHostToDevice, s));
            }
            out.push_back(c);
        }
    DF_CUDA(cudaStreamSynchronize(s));
    return out;
}

__global__ void add_kernel(const double* a, const double* b, long long n, double* c) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) c[i] = a[i] + b[i];
}

// zero the strictly upper triangle of a row-major square matrix
__global__ void zero_upper_kernel(double* M, int n) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    if (idx % n > idx / n) M[idx] = 0.0;
}

int fail(df_handle* h, const Error& e) {
    if (h) h->last_error = e.msg;
    return e.code;
}

}  // namespace

// Inverse of a lower-triangular block of at most 64 rows in place (row-major, leading dimension ld): the
// block is read into shared memory, then one thread per column j forward-substitutes and writes column j
// of the inverse (it reads back only values it wrote itself).
__global__ void tri_inv_small_kernel(double* __restrict__ L, int m, long long ld) {
    __shared__ double a[64][65];
    const int j = threadIdx.x;
    for (int r = 0; r < m; ++r)
        if (j < m) a[r][j] = L[(long long)r * ld + j];
    __syncthreads();
    if (j >= m) return;
    for (int i = 0; i < j; ++i) L[(long long)i * ld + j] = 0.0;
    L[(long long)j * ld + j] = 1.0 / a[j][j];
    for (int i = j + 1; i < m; ++i) {
        double t = 0.0;
        for (int k = j; k < i; ++k) t = fma(a[i][k], L[(long long)k * ld + j], t);
        L[(long long)i * ld + j] = -t / a[i][i];
    }
}

// Z <- L^-1 Z for a lower-triangular block of at most 64 rows (row-major, leading dimension ld) and the
// m x ncol right-hand sides Z (leading dimension ldz): one thread per column, forward substitution.
__global__ void tri_solve_small_kernel(const double* __restrict__ L, int m, long long ld, double* __restrict__ Z,
                                       int ncol, long long ldz) {
    __shared__ double a[64][65];
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) a[e / m][e % m] = L[(long long)(e / m) * ld + e % m];
    __syncthreads();
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncol) return;
    for (int i = 0; i < m; ++i) {
        double t = Z[(long long)i * ldz + j];
        for (int k = 0; k < i; ++k) t = fma(-a[i][k], Z[(long long)k * ldz + j], t);
        Z[(long long)i * ldz + j] = t / a[i][i];
    }
}

// Z <- L^-1 Z (L lower triangular m x m, leading dimension ld; Z m x ncol, leading dimension ldz) by
// recursion: Z1 <- L11^-1 Z1, Z2 <- Z2 - L21 Z1, Z2 <- L22^-1 Z2 (blocked forward substitution).
void tri_solve_lower(cudaStream_t s, const double* L, int m, long long ld, double* Z, int ncol, long long ldz) {
    if (m <= 64) {
        tri_solve_small_kernel<<<(ncol + 127) / 128, 128, 0, s>>>(L, m, ld, Z, ncol, ldz);
        DF_CHECK_LAUNCH();
        return;
    }
    const int m1 = ((m / 2 + 63) / 64) * 64, m2 = m - m1;
    tri_solve_lower(s, L, m1, ld, Z, ncol, ldz);
    dgemm(s, false, false, m2, ncol, m1, -1.0, L + (long long)m1 * ld, (int)ld, Z, (int)ldz, 1.0,
          Z + (long long)m1 * ldz, (int)ldz);
    tri_solve_lower(s, L + (long long)m1 * ld + m1, m2, ld, Z + (long long)m1 * ldz, ncol, ldz);
}

// L^-1 in place for lower-triangular L (m x m inside a row-major array of leading dimension ld; the
// upper triangle zero): with L = [[L11, 0], [L21, L22]], L^-1 = [[L11^-1, 0], [X21, L22^-1]] by recursion.
// X21 = -L22^-1 (L21 L11^-1) is taken by forward substitution with L22 before L22 is inverted: multiplying
// by the explicit L22^-1 instead left residuals |X L - I| a hundred times larger on an ill-conditioned
// metric (condition number 5e11 at 8 waters), enough to move the SCF energy by 1e-6 Eh. T is scratch
// of (m/2 + 64) x (m/2 + 64) doubles.
void tri_inv_lower(cudaStream_t s, double* L, int m, long long ld, double* T) {
    if (m <= 64) {
        tri_inv_small_kernel<<<1, 64, 0, s>>>(L, m, ld);
        DF_CHECK_LAUNCH();
        return;
    }
    const int m1 = ((m / 2 + 63) / 64) * 64, m2 = m - m1;
    double* L11 = L;
    double* L21 = L + (long long)m1 * ld;
    double* L22 = L21 + m1;
    tri_inv_lower(s, L11, m1, ld, T);
    dgemm(s, false, false, m2, m1, m1, -1.0, L21, (int)ld, L11, (int)ld, 0.0, T, m1);    // -L21 L11^-1
    tri_solve_lower(s, L22, m2, ld, T, m1, m1);                                         // X21 = L22^-1 T
    DF_CUDA(cudaMemcpy2DAsync(L21, sizeof(double) * ld, T, sizeof(double) * m1, sizeof(double) * m1, m2,
                              cudaMemcpyDeviceToDevice, s));
    tri_inv_lower(s, L22, m2, ld, T);
}

void build_B(df_handle* h, double tau, bool keep, int whitening) {
    cudaStream_t s = h->stream;
    const size_t rows = (size_t)h->naux * h->pk.row;
    cudaEvent_t ev[4];
    for (auto& e : ev) DF_CUDA(cudaEventCreate(&e));
    h->B.release();
    const bool have_3c = h->a3c_ready && h->A3c.p && h->A3c.n == rows;
    h->a3c_ready = false;
    if (!have_3c) {
        h->A3c.release();
        h->A3c.alloc(rows);
    }
    DF_CUDA(cudaEventRecord(ev[0], s));
    if (!have_3c) compute_three_center(h, h->A3c.p, tau);
    DF_CUDA(cudaEventRecord(ev[1], s));
    // metric Cholesky (P|Q) = L L^T: cuSOLVER works column-major, so the upper factor U (V = U^T U)
    // of the column-major matrix is the row-major lower factor L = U^T (trtri of U would give L^-1).
    const int na = h->naux;
    h->Linv.alloc((size_t)na * na);
    DF_CUDA(cudaMemcpyAsync(h->Linv.p, h->metric.p, sizeof(double) * na * na, cudaMemcpyDeviceToDevice, s));
    int lwork = 0;
    DF_SOLVER(cusolverDnDpotrf_bufferSize(h->solver, CUBLAS_FILL_MODE_UPPER, na, h->Linv.p, na, &lwork));
    double* work = nullptr;
    int* info = nullptr;
    DF_CUDA(cudaMalloc((void**)&work, sizeof(double) * std::max(lwork, 1)));
    DF_CUDA(cudaMalloc((void**)&info, sizeof(int)));
    int hinfo = 0;
    try {
        DF_CUDA(cudaStreamSynchronize(s));   // the integral kernels ahead on the stream are not potrf's time
        const auto tp0 = std::chrono::steady_clock::now();
        DF_SOLVER(cusolverDnDpotrf(h->solver, CUBLAS_FILL_MODE_UPPER, na, h->Linv.p, na, work, lwork, info));
        DF_CUDA(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
        DF_CUDA(cudaStreamSynchronize(s));
        if (hinfo != 0) throw Error{DF_E_NUMERIC, "metric (P|Q) is not positive definite (potrf info " + std::to_string(hinfo) + ")"};
        const auto tp1 = std::chrono::steady_clock::now();
        h->timings_ms[17] = std::chrono::duration<double, std::milli>(tp1 - tp0).count();   // potrf
        // the factor's inverse by blocks (FP64 products); DFHF_TRTRI=cusolver selects cuSOLVER's trtri, whose
        // first call in a process was measured at up to 0.9 s (4384 functions) against 0.08-0.14 s here
        const char* tri = std::getenv("DFHF_TRTRI");
        if (!(tri && std::string(tri) == "cusolver")) {
            // the row-major lower factor: zero its upper triangle, then invert by blocks
            zero_upper_kernel<<<(unsigned)(((long long)na * na + 255) / 256), 256, 0, s>>>(h->Linv.p, na);
            DF_CHECK_LAUNCH();
            DevBuf<double> T;
            T.alloc((size_t)((na / 2 + 63) / 64 * 64) * (size_t)(na / 2 + 64));
            tri_inv_lower(s, h->Linv.p, na, na, T.p);
            DF_CUDA(cudaStreamSynchronize(s));
        } else {
            size_t dws = 0, hws = 0;
            DF_SOLVER(cusolverDnXtrtri_bufferSize(h->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, na, CUDA_R_64F,
                                                  h->Linv.p, na, &dws, &hws));
            void* dbuf = nullptr;
            std::vector<char> hbuf(std::max<size_t>(hws, 1));
            DF_CUDA(cudaMalloc(&dbuf, std::max<size_t>(dws, 1)));
            cusolverStatus_t st = cusolverDnXtrtri(h->solver, CUBLAS_FILL_MODE_UPPER, CUBLAS_DIAG_NON_UNIT, na, CUDA_R_64F,
                                                   h->Linv.p, na, dbuf, dws, hbuf.data(), hws, info);
            DF_CUDA(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s));
            DF_CUDA(cudaStreamSynchronize(s));
            cudaFree(dbuf);
            if (st != CUSOLVER_STATUS_SUCCESS) throw Error{DF_E_CUDA, "cusolverDnXtrtri failed"};
        }
        h->timings_ms[18] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tp1).count();
        if (hinfo != 0) throw Error{DF_E_NUMERIC, "metric Cholesky factor is singular"};
    } catch (...) {
        cudaFree(work);
        cudaFree(info);
        throw;
    }
    cudaFree(work);
    cudaFree(info);
    zero_upper_kernel<<<(unsigned)(((long long)na * na + 255) / 256), 256, 0, s>>>(h->Linv.p, na);
    DF_CHECK_LAUNCH();
    DF_CUDA(cudaEventRecord(ev[2], s));
    const char* wenv = std::getenv("DFHF_WHITEN");
    if (whitening == DF_WHITEN_FP64) {
        // FP64 product on the FP64 pipe, in place by 64-row blocks of L^-1 (a copy first if A is kept)
        if (keep) {
            h->B.alloc(rows);
            DF_CUDA(cudaMemcpyAsync(h->B.p, h->A3c.p, sizeof(double) * rows, cudaMemcpyDeviceToDevice, s));
        } else {
            h->B.p = h->A3c.p;
            h->B.n = h->A3c.n;
            h->A3c.p = nullptr;
            h->A3c.n = 0;
        }
        whiten_fp64_inplace(s, na, h->pk.row, h->Linv.p, h->B.p, h->pk.row);
    } else if (wenv && std::string(wenv) == "ff") {
        // float-float whitening on the FP32 pipes (selectable for comparison)
        h->B.alloc(rows);
        DevBuf<double> lff;
        lff.alloc((size_t)na * na);
        whiten_float_float(s, na, h->pk.row, h->Linv.p, lff.p, h->A3c.p, h->B.p, h->pk.row, keep);
        DF_CUDA(cudaStreamSynchronize(s));
        lff.release();
    } else if (keep) {
        h->B.alloc(rows);
        whiten_ozaki(s, na, h->pk.row, h->pk.row, h->Linv.p, h->A3c.p, h->B.p);
    } else {
        // in place: the unwhitened tensor's memory becomes B
        whiten_ozaki(s, na, h->pk.row, h->pk.row, h->Linv.p, h->A3c.p, h->A3c.p);
        h->B.p = h->A3c.p;
        h->B.n = h->A3c.n;
        h->A3c.p = nullptr;
        h->A3c.n = 0;
    }
    DF_CUDA(cudaEventRecord(ev[3], s));
    DF_CUDA(cudaEventSynchronize(ev[3]));
    h->timings_ms[1] = elapsed_ms(ev[0], ev[1]);
    h->timings_ms[2] = elapsed_ms(ev[1], ev[2]);
    h->timings_ms[3] = elapsed_ms(ev[2], ev[3]);
    for (auto& e : ev) cudaEventDestroy(e);
    if (!keep) h->A3c.release();
    h->built = true;
    h->whitening = whitening;
}

// B for several handles: the three-centre integrals of all of them in one grouped launch per class (on
// the first handle's stream), then, if whiten_now, each handle's metric factor, inverse and whitening;
// otherwise the handles keep their integrals (a3c_ready) for build_B to finish later
void build_B_batch(df_handle** hs, int n, double tau, bool keep, int whitening, bool whiten_now) {
    std::vector<df_handle*> need;
    std::vector<double*> outs;
    for (int i = 0; i < n; ++i) {
        df_handle* h = hs[i];
        if (h->built) continue;
        h->B.release();
        h->A3c.release();
        h->A3c.alloc((size_t)h->naux * h->pk.row);
        h->a3c_ready = false;
        need.push_back(h);
        outs.push_back(h->A3c.p);
    }
    if (need.empty()) return;
    for (df_handle* h : need) DF_CUDA(cudaStreamSynchronize(h->stream));   // nothing queued reads A3c
    compute_three_center_grouped(need, outs, need[0]->stream);           // returns with the work done
    for (df_handle* h : need) h->a3c_ready = true;
    if (whiten_now)
        for (df_handle* h : need) build_B(h, tau, keep, whitening);
}

void jk_dispatch(df_handle* h, const double* dD, const double* dC, int nocc, double* dJ, double* dK, int precision,
                 int slices) {
    ensure_jk_buffers(h, nocc);
    coulomb_fp64(h, dD, dJ);
    const int ldy = ((nocc + 31) / 32) * 32;
    pad_occupied(h, dC, nocc, ldy);
    if (precision == DF_PREC_SPLIT)
        exchange_split(h, dC, nocc, slices, dK);
    else
        exchange_fp64(h, nocc, dK);
    h->timings_ms[16] = 6 + h->exchange_launches;   // J (pack, gamma, coulomb, split sum, unpack), pad C, K
}

// K alone for m columns of occupied-like coefficients dC (n x m, device), FP64 or split
void exchange_only(df_handle* h, const double* dC, int m, int precision, int slices, double* dK) {
    ensure_jk_buffers(h, m);
    if (precision == DF_PREC_SPLIT) {
        exchange_split(h, dC, m, slices, dK);
    } else {
        pad_occupied(h, dC, m, ((m + 31) / 32) * 32);
        exchange_fp64(h, m, dK);
    }
}

}  // namespace dfhf

using namespace dfhf;

extern "C" {

const char* df_strerror(int code) {
    switch (code) {
        case DF_OK: return "ok";
        case DF_E_ARG: return "invalid argument";
        case DF_E_NOMEM: return "device memory exhausted";
        case DF_E_CUDA: return "CUDA or cuSOLVER error";
        case DF_E_NOTCONV: return "SCF did not converge";
        case DF_E_STATE: return "call out of order";
        case DF_E_NUMERIC: return "numerical failure";
        case DF_E_TIMEOUT: return "device wait timed out";
        default: return "unknown error";
    }
}

const char* df_last_error(const df_handle* h) { return h ? h->last_error.c_str() : ""; }

int df_init(const df_atom* atoms, int natom, const df_shell* basis, int nbasis_sh, const df_shell* aux, int naux_sh,
            int charge, df_handle** out) {
    return dfhf::init_handle(atoms, natom, basis, nbasis_sh, aux, naux_sh, charge, out, true);
}

}  // extern "C"

// A handle for the system; closed_shell = false admits any electron count >= 1 (the atoms of the
// superposition-of-atomic-densities guess, whose SCF takes fractional occupations), with nocc the number
// of orbitals an Aufbau filling would touch, ceil(N / 2)
int dfhf::init_handle(const df_atom* atoms, int natom, const df_shell* basis, int nbasis_sh, const df_shell* aux,
                      int naux_sh, int charge, df_handle** out, bool closed_shell) {
    if (!out) return DF_E_ARG;
    *out = nullptr;
    if (!atoms || !basis || !aux || natom < 1 || nbasis_sh < 1 || naux_sh < 1) return DF_E_ARG;
    for (int i = 0; i < nbasis_sh; ++i)
        if (!(basis[i].exponent > 0) || basis[i].l < 0 || basis[i].l > DF_LMAX_ORB) return DF_E_ARG;
    for (int i = 0; i < naux_sh; ++i)
        if (!(aux[i].exponent > 0) || aux[i].l < 0 || aux[i].l > DF_LMAX_AUX) return DF_E_ARG;
    int zsum = 0;
    for (int i = 0; i < natom; ++i) {
        if (atoms[i].Z < 0) return DF_E_ARG;
        zsum += atoms[i].Z;
    }
    const int nelec = zsum - charge;
    if (closed_shell ? (nelec < 2 || nelec % 2) : nelec < 1) return DF_E_ARG;
    df_handle* h = new (std::nothrow) df_handle();
    if (!h) return DF_E_NOMEM;
    try {
        DF_CUDA(cudaGetDevice(&h->device));
        DF_CUDA(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
        h->stream = h->own_stream;
        DF_SOLVER(cusolverDnCreate(&h->solver));
        DF_SOLVER(cusolverDnSetStream(h->solver, h->stream));
        // df_coulomb_noalloc allocates nothing: its static scratch (address resolved here, which commits the
        // array's memory) and its kernels are made resident on the device now; without the scratch the
        // handle still works and that entry point reports why
        if (noalloc_scratch_address(&h->noalloc_scratch, &h->noalloc_error) != DF_OK) h->noalloc_scratch = nullptr;
        coulomb_kernels_load();
        h->atoms.assign(atoms, atoms + natom);
        h->basis.assign(basis, basis + nbasis_sh);
        h->aux.assign(aux, aux + naux_sh);
        for (auto& s : h->basis) h->n += 2 * s.l + 1;
        for (auto& s : h->aux) h->naux += 2 * s.l + 1;
        h->nelec = nelec;
        h->nocc = (nelec + 1) / 2;
        if (h->nocc > h->n) throw Error{DF_E_ARG, "more occupied orbitals than basis functions"};
        for (int i = 0; i < natom; ++i)
            for (int j = 0; j < i; ++j) {
                double r2 = 0;
                for (int d = 0; d < 3; ++d) r2 += (atoms[i].xyz[d] - atoms[j].xyz[d]) * (atoms[i].xyz[d] - atoms[j].xyz[d]);
                if (r2 == 0 && atoms[i].Z * atoms[j].Z != 0) throw Error{DF_E_ARG, "coincident nuclei"};
                if (r2 > 0) h->e_nuc += atoms[i].Z * atoms[j].Z / std::sqrt(r2);
            }
        Packing& pk = h->pk;
        pk.n = h->n;
        pk.nt = (h->n + TS - 1) / TS;
        pk.np = pk.nt * TS;
        pk.ntp = (long long)pk.nt * (pk.nt + 1) / 2;
        pk.row = pk.ntp * TS * TS;
        cudaStream_t s = h->stream;
        upload_shells(h->basis, h->dbas, s);
        upload_shells(h->aux, h->daux, s);
        h->pair_classes = make_pairs(h->basis, DF_LMAX_ORB, s);
        h->aux_pairs = make_pairs(h->aux, DF_LMAX_AUX, s);
        h->aux_by_l.assign(DF_LMAX_AUX + 1, {});
        for (int i = 0; i < naux_sh; ++i) h->aux_by_l[h->aux[i].l].push_back(i);
        for (int l = 0; l <= DF_LMAX_AUX; ++l)
            if (!h->aux_by_l[l].empty()) {
                h->d_aux_by_l[l].alloc(h->aux_by_l[l].size());
                DF_CUDA(cudaMemcpyAsync(h->d_aux_by_l[l].p, h->aux_by_l[l].data(), sizeof(int) * h->aux_by_l[l].size(),
                                        cudaMemcpyHostToDevice, s));
            }
        std::vector<double> axyz(3 * natom), aZ(natom);
        for (int i = 0; i < natom; ++i) {
            aZ[i] = atoms[i].Z;
            for (int d = 0; d < 3; ++d) axyz[3 * i + d] = atoms[i].xyz[d];
        }
        h->d_atom_xyz.alloc(3 * natom);
        h->d_atom_Z.alloc(natom);
        DF_CUDA(cudaMemcpyAsync(h->d_atom_xyz.p, axyz.data(), sizeof(double) * 3 * natom, cudaMemcpyHostToDevice, s));
        DF_CUDA(cudaMemcpyAsync(h->d_atom_Z.p, aZ.data(), sizeof(double) * natom, cudaMemcpyHostToDevice, s));
        const size_t nn = (size_t)h->n * h->n;
        h->S.alloc(nn);
        h->T.alloc(nn);
        h->V.alloc(nn);
        h->H.alloc(nn);
        h->metric.alloc((size_t)h->naux * h->naux);
        cudaEvent_t e0, e1;
        DF_CUDA(cudaEventCreate(&e0));
        DF_CUDA(cudaEventCreate(&e1));
        DF_CUDA(cudaEventRecord(e0, s));
        compute_one_electron(h);
        add_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(h->T.p, h->V.p, (long long)nn, h->H.p);
        DF_CHECK_LAUNCH();
        compute_metric(h);
        DF_CUDA(cudaEventRecord(e1, s));
        DF_CUDA(cudaEventSynchronize(e1));
        h->timings_ms[0] = elapsed_ms(e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    } catch (const Error& e) {
        int code = e.code;
        df_free(h);
        return code;
    } catch (const std::bad_alloc&) {
        df_free(h);
        return DF_E_NOMEM;
    }
    *out = h;
    return DF_OK;
}

extern "C" {

int df_sizes(const df_handle* h, int* n, int* naux, int* nocc, long long* packed_row) {
    if (!h) return DF_E_ARG;
    if (n) *n = h->n;
    if (naux) *naux = h->naux;
    if (nocc) *nocc = h->nocc;
    if (packed_row) *packed_row = h->pk.row;
    return DF_OK;
}

int df_build_B(df_handle* h, double screen_tau, int keep_3c) {
    return df_build_B_ex(h, screen_tau, keep_3c, DF_WHITEN_SPLIT);
}

int df_build_B_ex(df_handle* h, double screen_tau, int keep_3c, int whitening) {
    if (!h || screen_tau < 0 || (whitening != DF_WHITEN_SPLIT && whitening != DF_WHITEN_FP64)) return DF_E_ARG;
    try {
        DF_CUDA(cudaSetDevice(h->device));
        free_split(h);   // B slices cut from an earlier B are stale
        build_B(h, screen_tau, keep_3c != 0, whitening);
    } catch (const Error& e) {
        h->B.release();
        h->A3c.release();
        h->built = false;
        return fail(h, e);
    }
    return DF_OK;
}

int df_build_B_batch(df_handle** hs, int n, double screen_tau, int keep_3c, int whitening) {
    if (!hs || n < 1 || screen_tau < 0 || (whitening != DF_WHITEN_SPLIT && whitening != DF_WHITEN_FP64)) return DF_E_ARG;
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return DF_E_ARG;
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return DF_E_ARG;
        if (hs[i]->device != hs[0]->device) return DF_E_ARG;
    }
    try {
        DF_CUDA(cudaSetDevice(hs[0]->device));
        for (int i = 0; i < n; ++i) {
            free_split(hs[i]);
            hs[i]->built = false;
        }
        build_B_batch(hs, n, screen_tau, keep_3c != 0, whitening, true);
    } catch (const Error& e) {
        for (int i = 0; i < n; ++i) {
            hs[i]->last_error = e.msg;
            if (!hs[i]->built) {
                hs[i]->B.release();
                hs[i]->A3c.release();
                hs[i]->a3c_ready = false;
            }
        }
        return e.code;
    }
    return DF_OK;
}

int df_jk(df_handle* h, const double* D, const double* C_occ, int nocc, double* J, double* K, int device_ptrs,
          int precision, int slices) {
    if (!h || !D || !C_occ || !J || !K || nocc < 1 || nocc > h->n) return DF_E_ARG;
    if (precision != DF_PREC_FP64 && precision != DF_PREC_SPLIT) return DF_E_ARG;
    if (precision == DF_PREC_SPLIT && (slices < 2 || slices > 5)) return DF_E_ARG;
    if (!h->built) return fail(h, Error{DF_E_STATE, "df_jk before df_build_B"});
    try {
        DF_CUDA(cudaSetDevice(h->device));
        ensure_jk_buffers(h, nocc);
        const size_t nn = (size_t)h->n * h->n;
        cudaStream_t s = h->stream;
        const double *dD = D, *dC = C_occ;
        double *dJ = J, *dK = K;
        if (!device_ptrs) {
            DF_CUDA(cudaMemcpyAsync(h->dD.p, D, nn * sizeof(double), cudaMemcpyHostToDevice, s));
            DF_CUDA(cudaMemcpyAsync(h->dC.p, C_occ, (size_t)h->n * nocc * sizeof(double), cudaMemcpyHostToDevice, s));
            dD = h->dD.p;
            dC = h->dC.p;
            dJ = h->dJ.p;
            dK = h->dK.p;
        }
        jk_dispatch(h, dD, dC, nocc, dJ, dK, precision, slices);
        if (!device_ptrs) {
            DF_CUDA(cudaMemcpyAsync(J, dJ, nn * sizeof(double), cudaMemcpyDeviceToHost, s));
            DF_CUDA(cudaMemcpyAsync(K, dK, nn * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
        DF_CUDA(cudaStreamSynchronize(s));
    } catch (const Error& e) {
        return fail(h, e);
    }
    return DF_OK;
}

int scf_run(df_handle* h, const df_options* opts, df_result* out) {
    if (!h || !opts || !out) return DF_E_ARG;
    if (h->nelec % 2) return fail(h, Error{DF_E_STATE, "restricted Hartree-Fock needs an even electron count (scf_run_uhf)"});
    if (opts->max_iter < 1 || opts->conv_E <= 0 || opts->conv_err <= 0 || opts->screen_tau < 0 ||
        (opts->approx_diag != 0 && opts->approx_diag != 1) ||
        (opts->guess != DF_GUESS_CORE && opts->guess != DF_GUESS_SAD)) return DF_E_ARG;
    if (opts->precision != DF_PREC_FP64 && opts->precision != DF_PREC_SPLIT) return DF_E_ARG;
    if (opts->precision == DF_PREC_SPLIT && (opts->slices < 2 || opts->slices > 5)) return DF_E_ARG;
    try {
        DF_CUDA(cudaSetDevice(h->device));
        return scf_drive(h, opts, out);
    } catch (const Error& e) {
        out->status = e.code;
        return fail(h, e);
    }
}

int scf_run_guess(df_handle* h, const df_options* opts, const double* D0, df_result* out) {
    if (!h || !opts || !out) return DF_E_ARG;
    if (h->nelec % 2) return fail(h, Error{DF_E_STATE, "restricted Hartree-Fock needs an even electron count (scf_run_uhf)"});
    if (opts->max_iter < 1 || opts->conv_E <= 0 || opts->conv_err <= 0 || opts->screen_tau < 0 ||
        (opts->approx_diag != 0 && opts->approx_diag != 1) ||
        (opts->guess != DF_GUESS_CORE && opts->guess != DF_GUESS_SAD)) return DF_E_ARG;
    if (opts->precision != DF_PREC_FP64 && opts->precision != DF_PREC_SPLIT) return DF_E_ARG;
    if (opts->precision == DF_PREC_SPLIT && (opts->slices < 2 || opts->slices > 5)) return DF_E_ARG;
    try {
        DF_CUDA(cudaSetDevice(h->device));
        return scf_drive(h, opts, out, D0);
    } catch (const Error& e) {
        out->status = e.code;
        return fail(h, e);
    }
}

int scf_run_batch(df_handle** hs, int nmol, const df_options* opts, df_result* out) {
    if (!hs || nmol < 1 || !opts || !out) return DF_E_ARG;
    if (opts->max_iter < 1 || opts->conv_E <= 0 || opts->conv_err <= 0 || opts->screen_tau < 0 ||
        (opts->approx_diag != 0 && opts->approx_diag != 1) ||
        (opts->guess != DF_GUESS_CORE && opts->guess != DF_GUESS_SAD)) return DF_E_ARG;
    if (opts->precision != DF_PREC_FP64 && opts->precision != DF_PREC_SPLIT) return DF_E_ARG;
    if (opts->precision == DF_PREC_SPLIT && (opts->slices < 2 || opts->slices > 5)) return DF_E_ARG;
    int dev = -1;
    for (int i = 0; i < nmol; ++i) {
        if (!hs[i]) return DF_E_ARG;
        if (hs[i]->nelec % 2) return DF_E_STATE;   // restricted Hartree-Fock: even electron counts only
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return DF_E_ARG;   // each molecule needs its own handle
        if (dev < 0) dev = hs[i]->device;
        if (hs[i]->device != dev) return DF_E_ARG;
    }
    try {
        DF_CUDA(cudaSetDevice(dev));
        return scf_drive_batch(hs, nmol, opts, out);
    } catch (const Error& e) {
        for (int i = 0; i < nmol; ++i) {
            hs[i]->last_error = e.msg;
            if (out[i].status == 0 && !out[i].converged) out[i].status = e.code;
        }
        return e.code;
    }
}

int df_init_open(const df_atom* atoms, int natom, const df_shell* basis, int nbasis_sh, const df_shell* aux,
                 int naux_sh, int charge, df_handle** out) {
    return dfhf::init_handle(atoms, natom, basis, nbasis_sh, aux, naux_sh, charge, out, false);
}

int scf_run_uhf(df_handle* h, const df_options* opts, int nalpha, int nbeta, df_result* out) {
    if (!h || !opts || !out) return DF_E_ARG;
    if (opts->max_iter < 1 || opts->conv_E <= 0 || opts->conv_err <= 0 || opts->screen_tau < 0) return DF_E_ARG;
    if (opts->precision != DF_PREC_FP64 && opts->precision != DF_PREC_SPLIT) return DF_E_ARG;
    if (opts->precision == DF_PREC_SPLIT && (opts->slices < 2 || opts->slices > 5)) return DF_E_ARG;
    if ((opts->guess != DF_GUESS_CORE && opts->guess != DF_GUESS_SPIN) || opts->incremental || opts->approx_diag)
        return fail(h, Error{DF_E_ARG, "scf_run_uhf: core-Hamiltonian or spin-density guess, full builds and full "
                                       "eigensolves only"});
    if (nalpha < nbeta || nbeta < 0 || nalpha + nbeta != h->nelec || nalpha > h->n)
        return fail(h, Error{DF_E_ARG, "scf_run_uhf: need nalpha >= nbeta >= 0, nalpha + nbeta = electron count"});
    if (opts->guess == DF_GUESS_SPIN && !h->Dspin.p)
        return fail(h, Error{DF_E_STATE, "scf_run_uhf: no spin densities of an earlier open-shell run on this handle"});
    try {
        DF_CUDA(cudaSetDevice(h->device));
        return scf_drive_uhf(h, opts, nalpha, nbeta, out);
    } catch (const Error& e) {
        out->status = e.code;
        return fail(h, e);
    }
}

int scf_run_rohf(df_handle* h, const df_options* opts, int nalpha, int nbeta, double level_shift, df_result* out) {
    if (!h || !opts || !out) return DF_E_ARG;
    if (opts->max_iter < 1 || opts->conv_E <= 0 || opts->conv_err <= 0 || opts->screen_tau < 0) return DF_E_ARG;
    if (opts->precision != DF_PREC_FP64 && opts->precision != DF_PREC_SPLIT) return DF_E_ARG;
    if (opts->precision == DF_PREC_SPLIT && (opts->slices < 2 || opts->slices > 5)) return DF_E_ARG;
    if (!(level_shift >= 0.0) || !std::isfinite(level_shift))
        return fail(h, Error{DF_E_ARG, "scf_run_rohf: the level shift must be finite and >= 0"});
    if (opts->guess != DF_GUESS_CORE || opts->incremental || opts->approx_diag)
        return fail(h, Error{DF_E_ARG, "scf_run_rohf: core-Hamiltonian guess, full builds and full eigensolves only"});
    if (nalpha < nbeta || nbeta < 0 || nalpha + nbeta != h->nelec || nalpha > h->n)
        return fail(h, Error{DF_E_ARG, "scf_run_rohf: need nalpha >= nbeta >= 0, nalpha + nbeta = electron count"});
    try {
        DF_CUDA(cudaSetDevice(h->device));
        return scf_drive_rohf(h, opts, nalpha, nbeta, level_shift, out);
    } catch (const Error& e) {
        out->status = e.code;
        return fail(h, e);
    }
}

int df_get_rows(df_handle* h, int which, int p0, int count, double* out) {
    if (!h || !out || p0 < 0 || count < 1 || p0 + count > h->naux || (which != 0 && which != 1)) return DF_E_ARG;
    const double* src = which == 0 ? h->A3c.p : h->B.p;
    if (!src) return fail(h, Error{DF_E_STATE, which == 0 ? "unwhitened tensor not kept" : "B not built"});
    try {
        const size_t nn = (size_t)h->n * h->n;
        DevBuf<double> tmp;
        tmp.alloc(nn * count);
        unpack_rows(h, src, p0, count, tmp.p);
        DF_CUDA(cudaMemcpyAsync(out, tmp.p, nn * count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        DF_CUDA(cudaStreamSynchronize(h->stream));
        tmp.release();
    } catch (const Error& e) {
        return fail(h, e);
    }
    return DF_OK;
}

int df_get_matrix(df_handle* h, int which, double* out) {
    if (!h || !out) return DF_E_ARG;
    const size_t nn = (size_t)h->n * h->n, aa = (size_t)h->naux * h->naux;
    const double* src = nullptr;
    size_t count = nn;
    switch (which) {
        case 0: src = h->S.p; break;
        case 1: src = h->T.p; break;
        case 2: src = h->V.p; break;
        case 3: src = h->H.p; break;
        case 4: src = h->metric.p; count = aa; break;
        case 5: src = h->Linv.p; count = aa; break;
        case 6: src = h->Dm.p; break;
        case 7: src = h->F.p; break;
        case 8: src = h->dJ.p; break;
        case 9: src = h->dK.p; break;
        case 10: src = h->C.p; count = (size_t)h->n * h->nX; break;
        case 11: src = h->eps.p; count = h->n; break;
        case 12: src = h->Dspin.p; break;                             // UHF alpha density
        case 13: src = h->Dspin.p ? h->Dspin.p + nn : nullptr; break;   // UHF beta density
        default: return DF_E_ARG;
    }
    if (!src) return fail(h, Error{DF_E_STATE, "matrix not available yet"});
    try {
        if (which == 10 && h->nX < h->n) {   // pad dropped orbitals with zero columns
            std::vector<double> tmp((size_t)h->n * h->nX);
            DF_CUDA(cudaMemcpy(tmp.data(), src, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost));
            for (int r = 0; r < h->n; ++r)
                for (int c = 0; c < h->n; ++c) out[(size_t)r * h->n + c] = c < h->nX ? tmp[(size_t)r * h->nX + c] : 0.0;
            return DF_OK;
        }
        DF_CUDA(cudaStreamSynchronize(h->stream));
        DF_CUDA(cudaMemcpy(out, src, count * sizeof(double), cudaMemcpyDeviceToHost));
    } catch (const Error& e) {
        return fail(h, e);
    }
    return DF_OK;
}

int df_rint_pow2(const double* v, const int* k, long long count, long long* out) {
    if (count < 0 || (count > 0 && (!v || !k || !out))) return DF_E_ARG;
    for (long long i = 0; i < count; ++i) out[i] = dfhf::rint_pow2(v[i], k[i]);
    return DF_OK;
}

int df_rys(const double* T, int count, int nroots, double* x, double* w) {
    if (!T || !x || !w || count < 1 || nroots < 1 || nroots > 4) return DF_E_ARG;
    try {
        double *dT = nullptr, *dx = nullptr, *dw = nullptr;
        DF_CUDA(cudaMalloc((void**)&dT, sizeof(double) * count));
        DF_CUDA(cudaMalloc((void**)&dx, sizeof(double) * count * nroots));
        DF_CUDA(cudaMalloc((void**)&dw, sizeof(double) * count * nroots));
        DF_CUDA(cudaMemcpy(dT, T, sizeof(double) * count, cudaMemcpyHostToDevice));
        rys_eval(dT, count, nroots, dx, dw, 0);
        DF_CUDA(cudaMemcpy(x, dx, sizeof(double) * count * nroots, cudaMemcpyDeviceToHost));
        DF_CUDA(cudaMemcpy(w, dw, sizeof(double) * count * nroots, cudaMemcpyDeviceToHost));
        cudaFree(dT);
        cudaFree(dx);
        cudaFree(dw);
    } catch (const Error& e) {
        return e.code;
    }
    return DF_OK;
}

int df_scf_history(const df_handle* h, double* out, int max_rows) {
    if (!h || (!out && max_rows > 0) || max_rows < 0) return DF_E_ARG;
    const int rows = (int)(h->history.size() / 6);
    const int n = rows < max_rows ? rows : max_rows;
    for (int i = 0; i < 6 * n; ++i) out[i] = h->history[i];
    return rows;
}

int df_prepare(void) {
    try {
        rys_table_host();
    } catch (const Error& e) {
        return e.code;
    }
    return DF_OK;
}

int df_set_stream(df_handle* h, void* stream) {
    if (!h) return DF_E_ARG;
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
    if (cusolverDnSetStream(h->solver, h->stream) != CUSOLVER_STATUS_SUCCESS) return DF_E_CUDA;
    return DF_OK;
}

int df_timings(const df_handle* h, double* ms, int count) {
    if (!h || !ms || count < 0) return DF_E_ARG;
    for (int i = 0; i < count && i < 20; ++i) ms[i] = h->timings_ms[i];
    return DF_OK;
}

void df_free(df_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_split(h);
    free_shells(h->dbas);
    free_shells(h->daux);
    for (auto& c : h->pair_classes) cudaFree(c.d_pairs);
    for (auto& c : h->aux_pairs) cudaFree(c.d_pairs);
    if (h->solver) cusolverDnDestroy(h->solver);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    // device buffers released here, while the handle's device is current (their destructors then find them empty)
    DevBuf<double>* bufs[] = {&h->d_atom_xyz, &h->d_atom_Z, &h->S, &h->T, &h->V, &h->H, &h->metric, &h->Linv,
                              &h->A3c, &h->B, &h->Dw, &h->gamma, &h->Jp, &h->Y, &h->Kpart, &h->Cpad, &h->dD,
                              &h->dC, &h->dJ, &h->dK, &h->X, &h->F, &h->Fx, &h->Dm, &h->C, &h->eps, &h->work1,
                              &h->work2, &h->work3, &h->diisF, &h->diisE, &h->diisB, &h->Dspin};
    for (auto* b : bufs) b->release();
    h->ktiles.release();
    for (auto& b : h->d_aux_by_l) b.release();
    delete h;
}

}  // extern "C"
