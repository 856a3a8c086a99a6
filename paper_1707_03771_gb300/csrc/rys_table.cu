// Host construction of the Rys root/weight tables used by rys.cuh, and the df_rys test hook.
//
// Gauss rule of the measure dmu_T(x) = exp(-T x) x^{-1/2} dx / 2 on [0,1] (x = t^2), whose moments
// are the Boys functions F_k(T):
//  1. discretise mu_T by composite Gauss-Legendre quadrature in t (64 panels x 16 nodes);
//  2. Stieltjes procedure on the discrete measure -> recurrence coefficients alpha_k, beta_k of the
//     monic orthogonal polynomials (Gautschi, "Orthogonal Polynomials: Computation and
//     Approximation", 2004, section 2.2.3);
//  3. Golub-Welsch: nodes = eigenvalues of the Jacobi matrix, weights = beta_0 v_0^2
//     (Golub & Welsch, Math. Comp. 23, 221 (1969)); eigenpairs by cyclic Jacobi rotations.
// Everything in long double. Nodes and weights are then fitted by Chebyshev series on unit
// intervals of T, and the fit is checked against the directly computed moments before use.
// For T >= 60 the rule is generalised Gauss-Laguerre with alpha = -1/2 (monic recurrence
// alpha_k = 2k + 1/2, beta_k = k (k - 1/2), beta_0 = Gamma(1/2)).
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <unistd.h>

#include "common.cuh"
#include "rys.cuh"

namespace dfhf {

namespace {

typedef long double ld;

void gauss_legendre(int n, std::vector<ld>& x, std::vector<ld>& w) {
    x.resize(n);
    w.resize(n);
    const ld pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        ld z = std::cos(pi * (i + 0.75L) / (n + 0.5L)), dp = 0;
        for (int it = 0; it < 100; ++it) {
            ld p0 = 1, p1 = z;
            for (int k = 2; k <= n; ++k) {
                ld p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1);
            ld dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-19L) break;
        }
        ld p0 = 1, p1 = z;
        for (int k = 2; k <= n; ++k) {
            ld p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1);
        x[i] = z;
        w[i] = 2 / ((1 - z * z) * dp * dp);
    }
}

// symmetric eigen-decomposition by cyclic Jacobi rotations; V columns are eigenvectors
void jacobi_eigen(int n, ld* A, ld* V) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + j] = (i == j);
    for (int sweep = 0; sweep < 100; ++sweep) {
        ld off = 0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
        if (off < 1e-40L) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                ld apq = A[p * n + q];
                if (std::fabs(apq) < 1e-300L) continue;
                ld theta = (A[q * n + q] - A[p * n + p]) / (2 * apq);
                ld t = (theta >= 0 ? 1 : -1) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
                ld c = 1 / std::sqrt(t * t + 1), s = t * c;
                for (int k = 0; k < n; ++k) {
                    ld akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    ld apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    ld vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
}

// Golub-Welsch from recurrence coefficients; nodes ascending
void golub_welsch(int n, const ld* alpha, const ld* beta, ld* x, ld* w) {
    ld A[16], V[16];
    for (int i = 0; i < n * n; ++i) A[i] = 0;
    for (int i = 0; i < n; ++i) A[i * n + i] = alpha[i];
    for (int i = 1; i < n; ++i) A[i * n + i - 1] = A[(i - 1) * n + i] = std::sqrt(beta[i]);
    jacobi_eigen(n, A, V);
    std::vector<std::pair<ld, ld>> nw(n);
    for (int i = 0; i < n; ++i) nw[i] = {A[i * n + i], beta[0] * V[i] * V[i]};
    std::sort(nw.begin(), nw.end());
    for (int i = 0; i < n; ++i) {
        x[i] = nw[i].first;
        w[i] = nw[i].second;
    }
}

struct Discrete {
    std::vector<ld> t, g;   // composite Gauss-Legendre in t on [0,1]
    Discrete() {
        std::vector<ld> gx, gw;
        gauss_legendre(16, gx, gw);
        const int panels = 64;
        for (int p = 0; p < panels; ++p) {
            ld a = (ld)p / panels, b = (ld)(p + 1) / panels;
            for (int q = 0; q < 16; ++q) {
                t.push_back((a + b) / 2 + (b - a) / 2 * gx[q]);
                g.push_back((b - a) / 2 * gw[q]);
            }
        }
    }
    // Gauss rule of mu_T with n nodes (Stieltjes on the discrete measure)
    void rule(int n, ld T, ld* x, ld* w, ld* moments /* 2n, may be null */) const {
        const size_t N = t.size();
        std::vector<ld> xs(N), ws(N), pm(N, 0), p(N, 1), pn(N);
        for (size_t j = 0; j < N; ++j) {
            xs[j] = t[j] * t[j];
            ws[j] = g[j] * std::exp(-T * xs[j]);
        }
        if (moments)
            for (int k = 0; k < 2 * n; ++k) {
                ld s = 0;
                for (size_t j = 0; j < N; ++j) s += ws[j] * std::pow(xs[j], (ld)k);
                moments[k] = s;
            }
        ld alpha[RYS_NMAX], beta[RYS_NMAX], prev = 0;
        for (int k = 0; k < n; ++k) {
            ld num = 0, den = 0;
            for (size_t j = 0; j < N; ++j) {
                num += ws[j] * xs[j] * p[j] * p[j];
                den += ws[j] * p[j] * p[j];
            }
            alpha[k] = num / den;
            beta[k] = (k == 0) ? den : den / prev;
            prev = den;
            for (size_t j = 0; j < N; ++j) pn[j] = (xs[j] - alpha[k]) * p[j] - (k > 0 ? beta[k] * pm[j] : 0);
            pm.swap(p);
            p.swap(pn);
        }
        golub_welsch(n, alpha, beta, x, w);
    }
};

std::vector<double> build_table() {
    std::vector<double> tab(RYS_TABLE_SIZE, 0.0);
    Discrete disc;
    const ld pi = 3.141592653589793238462643383279502884L;
    for (int n = 1; n <= RYS_NMAX; ++n) {
        for (int k = 0; k < RYS_NINT; ++k) {
            std::vector<ld> vals((size_t)RYS_NC * 2 * n);   // [node j][function f]
            for (int j = 0; j < RYS_NC; ++j) {
                ld s = std::cos(pi * (j + 0.5L) / RYS_NC);
                ld T = k + (s + 1) / 2;
                ld x[RYS_NMAX], w[RYS_NMAX];
                disc.rule(n, T, x, w, nullptr);
                for (int i = 0; i < n; ++i) {
                    vals[(size_t)j * 2 * n + i] = x[i];
                    vals[(size_t)j * 2 * n + n + i] = w[i];
                }
            }
            double* c = tab.data() + rys_offset(n) + (size_t)k * 2 * n * RYS_NC;
            for (int f = 0; f < 2 * n; ++f)
                for (int m = 0; m < RYS_NC; ++m) {
                    ld s = 0;
                    for (int j = 0; j < RYS_NC; ++j)
                        s += vals[(size_t)j * 2 * n + f] * std::cos(pi * m * (j + 0.5L) / RYS_NC);
                    s *= 2.0L / RYS_NC;
                    if (m == 0) s /= 2;
                    c[f * RYS_NC + m] = (double)s;
                }
        }
        // generalised Gauss-Laguerre, alpha = -1/2
        ld alpha[RYS_NMAX], beta[RYS_NMAX], x[RYS_NMAX], w[RYS_NMAX];
        for (int k = 0; k < n; ++k) {
            alpha[k] = 2 * k + 0.5L;
            beta[k] = (k == 0) ? std::sqrt(pi) : k * (k - 0.5L);
        }
        golub_welsch(n, alpha, beta, x, w);
        double* a = tab.data() + RYS_ASYM + n * (n - 1);
        for (int i = 0; i < n; ++i) {
            a[i] = (double)x[i];
            a[n + i] = (double)(w[i] / 2);
        }
    }
    // validate: interpolated rules reproduce the moments of mu_T
    double worst = 0;
    for (int n = 1; n <= RYS_NMAX; ++n)
        for (int s = 0; s < 400; ++s) {
            double T = (s < 390) ? 0.1537 * s + 1e-3 * (s % 7) : 60.0 + 13.0 * (s - 390);
            ld mom[2 * RYS_NMAX];
            ld xx[RYS_NMAX], ww[RYS_NMAX];
            disc.rule(n, T, xx, ww, mom);
            double x[RYS_NMAX], w[RYS_NMAX];
            switch (n) {
                case 1: rys_roots<1>(T, tab.data(), x, w); break;
                case 2: rys_roots<2>(T, tab.data(), x, w); break;
                case 3: rys_roots<3>(T, tab.data(), x, w); break;
                default: rys_roots<4>(T, tab.data(), x, w); break;
            }
            for (int k = 0; k < 2 * n; ++k) {
                ld q = 0;
                for (int i = 0; i < n; ++i) q += (ld)w[i] * std::pow((ld)x[i], (ld)k);
                worst = std::max(worst, (double)(std::fabs(q - mom[k]) / mom[k]));
            }
        }
    if (!(worst < 5e-14))
        throw Error{DF_E_NUMERIC, "Rys table self-check failed: max relative moment error " + std::to_string(worst)};
    return tab;
}

std::mutex g_mu;
std::vector<double> g_host;
std::map<int, double*> g_dev;

// The table takes seconds to build where long double is emulated in software, so the validated
// table is cached beside the library: 8-byte magic, entry count, the doubles, FNV-1a of their bytes.
const char kMagic[8] = {'D', 'F', 'R', 'Y', 'S', '0', '0', '1'};

uint64_t fnv1a(const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    uint64_t h = 1469598103934665603ULL;
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ULL;
    return h;
}

std::string cache_path() {
    if (const char* env = std::getenv("DFHF_TABLE_CACHE")) return env;
    Dl_info info;
    if (dladdr((void*)&fnv1a, &info) && info.dli_fname) {
        std::string f = info.dli_fname;
        size_t slash = f.rfind('/');
        return (slash == std::string::npos ? std::string(".") : f.substr(0, slash)) + "/rys_table.bin";
    }
    return "";
}

bool load_cache(const std::string& path, std::vector<double>& out) {
    if (path.empty()) return false;
    FILE* f = std::fopen(path.c_str(), "rb");
    if (!f) return false;
    char magic[8];
    long long count = 0;
    uint64_t sum = 0;
    std::vector<double> v(RYS_TABLE_SIZE);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(&count, sizeof(count), 1, f) == 1 && count == RYS_TABLE_SIZE &&
              std::fread(v.data(), sizeof(double), v.size(), f) == v.size() && std::fread(&sum, sizeof(sum), 1, f) == 1 &&
              sum == fnv1a(v.data(), v.size() * sizeof(double));
    std::fclose(f);
    if (ok) out.swap(v);
    return ok;
}

void store_cache(const std::string& path, const std::vector<double>& v) {
    if (path.empty()) return;
    std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;
    long long count = (long long)v.size();
    uint64_t sum = fnv1a(v.data(), v.size() * sizeof(double));
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&count, sizeof(count), 1, f) == 1 &&
              std::fwrite(v.data(), sizeof(double), v.size(), f) == v.size() && std::fwrite(&sum, sizeof(sum), 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    if (ok) std::rename(tmp.c_str(), path.c_str());
    else std::remove(tmp.c_str());
}

}  // namespace

const double* rys_table_host() {
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_host.empty()) {
        const std::string path = cache_path();
        if (!load_cache(path, g_host)) {
            g_host = build_table();
            store_cache(path, g_host);
        }
    }
    return g_host.data();
}

const double* rys_table_device() {
    const double* host = rys_table_host();
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    DF_CUDA(cudaGetDevice(&dev));
    auto it = g_dev.find(dev);
    if (it != g_dev.end()) return it->second;
    double* d = nullptr;
    DF_CUDA(cudaMalloc((void**)&d, RYS_TABLE_SIZE * sizeof(double)));
    DF_CUDA(cudaMemcpy(d, host, RYS_TABLE_SIZE * sizeof(double), cudaMemcpyHostToDevice));
    g_dev[dev] = d;
    return d;
}

template <int N>
__global__ void rys_eval_kernel(const double* T, int count, const double* tab, double* x, double* w) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double xr[N], wr[N];
    rys_roots<N>(T[i], tab, xr, wr);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        x[(size_t)i * N + k] = xr[k];
        w[(size_t)i * N + k] = wr[k];
    }
}

void rys_eval(const double* dT, int count, int n, double* dx, double* dw, cudaStream_t s) {
    const double* tab = rys_table_device();
    int blocks = (count + 127) / 128;
    switch (n) {
        case 1: rys_eval_kernel<1><<<blocks, 128, 0, s>>>(dT, count, tab, dx, dw); break;
        case 2: rys_eval_kernel<2><<<blocks, 128, 0, s>>>(dT, count, tab, dx, dw); break;
        case 3: rys_eval_kernel<3><<<blocks, 128, 0, s>>>(dT, count, tab, dx, dw); break;
        case 4: rys_eval_kernel<4><<<blocks, 128, 0, s>>>(dT, count, tab, dx, dw); break;
        default: throw Error{DF_E_ARG, "df_rys: n must be in 1..4"};
    }
    DF_CHECK_LAUNCH();
}

}  // namespace dfhf
