// Learned initial guess: a small MLP maps rotation-invariant features of each water's environment to
// the water's 50 x 50 diagonal density block expressed in the molecule's own frame; the blocks are
// rotated to the laboratory frame with real-solid-harmonic rotation matrices (l <= 2) and assembled
// block-diagonally into D0. A second network maps features of each ordered pair of waters within a cutoff
// (the second water's atoms in the first one's frame, atom-pair distances) to the pair's 50 x 50
// off-diagonal block in the first water's frame. The SCF then starts from the natural orbitals of D0
// (scf_run_guess).
// Training (forward, backward, Adam) and BF16 inference run in this file's CUDA kernels.
// The paper has no learned guess; this is the build's design (its quality is a measured outcome).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "common.cuh"

struct df_mlp {
    int nin = 0, nh = 0, nlayers = 0, nout = 0;   // nlayers hidden layers of width nh
    std::vector<int> dims;                        // nin, nh, ..., nh, nout
    std::vector<long long> woff, boff;            // offsets of W_l (out x in) and b_l in params
    long long nparams = 0;
    dfhf::DevBuf<float> P, G, Mom, Vel;           // parameters, gradients, Adam moments
    dfhf::DevBuf<__nv_bfloat16> Pbf;              // BF16 copy for inference
    int adam_t = 0;
    cudaStream_t stream = nullptr;
};

namespace dfhf {

namespace {

// ---------------------------------------------------------------------------------------------
// FP32 GEMM: C = alpha op(A) op(B) + beta C, row-major (64 x 64 tiles, 4 x 4 per thread)
// ---------------------------------------------------------------------------------------------
constexpr int FBM = 64, FBN = 64, FBK = 16;
__global__ void __launch_bounds__(256) sgemm_kernel(bool ta, bool tb, int m, int n, int k, float alpha,
                                                    const float* __restrict__ A, int lda, const float* __restrict__ B,
                                                    int ldb, float beta, float* __restrict__ C, int ldc) {
    __shared__ float As[FBK][FBM + 1];
    __shared__ float Bs[FBK][FBN + 1];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * FBM, n0 = blockIdx.x * FBN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < k; k0 += FBK) {
        for (int idx = tid; idx < FBM * FBK; idx += 256) {
            const int r = ta ? idx % FBM : idx / FBK, c = ta ? idx / FBM : idx % FBK;
            const int gm = m0 + r, gk = k0 + c;
            As[c][r] = (gm < m && gk < k) ? (ta ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk]) : 0.f;
        }
        for (int idx = tid; idx < FBK * FBN; idx += 256) {
            const int r = tb ? idx % FBK : idx / FBN, c = tb ? idx / FBK : idx % FBN;
            const int gk = k0 + r, gn = n0 + c;
            Bs[r][c] = (gk < k && gn < n) ? (tb ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < FBK; ++kk)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(As[kk][ty + 16 * i], Bs[kk][tx + 16 * j], acc[i][j]);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
            if (gm < m && gn < n) {
                float* c = C + (long long)gm * ldc + gn;
                *c = alpha * acc[i][j] + (beta == 0.f ? 0.f : beta * *c);
            }
        }
}

void sgemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, float alpha, const float* A, int lda, const float* B,
           int ldb, float beta, float* C, int ldc) {
    dim3 grid((n + FBN - 1) / FBN, (m + FBM - 1) / FBM);
    sgemm_kernel<<<grid, 256, 0, s>>>(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    DF_CHECK_LAUNCH();
}

// Z[r][c] += b[c]; A = relu(Z) (hidden) or Z (output)
__global__ void bias_act_kernel(float* __restrict__ Z, const float* __restrict__ b, int rows, int cols, bool relu,
                                float* __restrict__ A) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * cols) return;
    const float z = Z[i] + b[i % cols];
    Z[i] = z;
    A[i] = relu ? fmaxf(z, 0.f) : z;
}

// dZ = dA * relu'(Z)
__global__ void relu_back_kernel(const float* __restrict__ Z, float* __restrict__ dA, long long len) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len && Z[i] <= 0.f) dA[i] = 0.f;
}

// db[c] = sum_r dZ[r][c]
__global__ void colsum_kernel(const float* __restrict__ dZ, int rows, int cols, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dZ[(long long)r * cols + c];
    db[c] = s;
}

// dY = 2 (Yp - Y) / (rows cols); loss partials per block (deterministic two-stage sum)
__global__ void mse_kernel(const float* __restrict__ Yp, const float* __restrict__ Y, long long len, float scale,
                           float* __restrict__ dY, float* __restrict__ part) {
    __shared__ float sm[256];
    float s = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
        const float d = Yp[i] - Y[i];
        dY[i] = 2.f * d * scale;
        s += d * d;
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0] * scale;
}

// Adam (Kingma & Ba 2015) with bias correction
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void to_bf16_kernel(const float* __restrict__ x, long long n, __nv_bfloat16* __restrict__ y) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// BF16 inference layer: out[r][o] = act(sum_i in[r][i] W[o][i] + b[o]) with BF16 inputs and weights,
// FP32 accumulation; one warp per output element (inputs re-rounded to BF16 between layers)
__global__ void bf16_layer_kernel(const __nv_bfloat16* __restrict__ in, int rows, int nin,
                                  const __nv_bfloat16* __restrict__ W, const __nv_bfloat16* __restrict__ b, int nout,
                                  bool relu, __nv_bfloat16* __restrict__ out_bf, float* __restrict__ out_f) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (long long)rows * nout) return;
    const int r = (int)(w / nout), o = (int)(w % nout);
    float s = 0.f;
    for (int i = lane; i < nin; i += 32)
        s = fmaf(__bfloat162float(in[(long long)r * nin + i]), __bfloat162float(W[(long long)o * nin + i]), s);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
        s += __bfloat162float(b[o]);
        if (relu) s = fmaxf(s, 0.f);
        if (out_bf) out_bf[(long long)r * nout + o] = __float2bfloat16_rn(s);
        if (out_f) out_f[(long long)r * nout + o] = s;
    }
}

inline unsigned nb(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

int fail_code(df_handle* h, const Error& e) {
    h->last_error = e.msg;
    return e.code;
}

// forward of the FP32 network over `rows` samples; Zs/As hold every layer's pre/post activations
void forward(df_mlp* m, const float* X, int rows, std::vector<float*>& Zs, std::vector<float*>& As) {
    const int L = (int)m->dims.size() - 1;
    const float* in = X;
    for (int l = 0; l < L; ++l) {
        const int ni = m->dims[l], no = m->dims[l + 1];
        sgemm(m->stream, false, true, rows, no, ni, 1.f, in, ni, m->P.p + m->woff[l], ni, 0.f, Zs[l], no);
        bias_act_kernel<<<nb((long long)rows * no), 256, 0, m->stream>>>(Zs[l], m->P.p + m->boff[l], rows, no, l < L - 1,
                                                                        As[l]);
        DF_CHECK_LAUNCH();
        in = As[l];
    }
}

struct Work {
    std::vector<DevBuf<float>> Z, A, dA;
    DevBuf<float> dY, part;
    void alloc(df_mlp* m, int rows) {
        const int L = (int)m->dims.size() - 1;
        Z.resize(L);
        A.resize(L);
        dA.resize(L);
        for (int l = 0; l < L; ++l) {
            Z[l].alloc((size_t)rows * m->dims[l + 1]);
            A[l].alloc((size_t)rows * m->dims[l + 1]);
            dA[l].alloc((size_t)rows * m->dims[l + 1]);
        }
        dY.alloc((size_t)rows * m->nout);
        part.alloc(256);
    }
    void release() {
        for (auto& b : Z) b.release();
        for (auto& b : A) b.release();
        for (auto& b : dA) b.release();
        dY.release();
        part.release();
    }
};

// loss and gradient (into m->G) over one batch; returns the loss (synchronises)
float loss_and_grad(df_mlp* m, const float* X, const float* Y, int rows, Work& w) {
    const int L = (int)m->dims.size() - 1;
    std::vector<float*> Zs(L), As(L);
    for (int l = 0; l < L; ++l) {
        Zs[l] = w.Z[l].p;
        As[l] = w.A[l].p;
    }
    forward(m, X, rows, Zs, As);
    const long long len = (long long)rows * m->nout;
    const float scale = 1.f / (float)len;
    mse_kernel<<<256, 256, 0, m->stream>>>(As[L - 1], Y, len, scale, w.dA[L - 1].p, w.part.p);
    DF_CHECK_LAUNCH();
    for (int l = L - 1; l >= 0; --l) {
        const int ni = m->dims[l], no = m->dims[l + 1];
        float* dZ = w.dA[l].p;
        if (l < L - 1) {
            relu_back_kernel<<<nb((long long)rows * no), 256, 0, m->stream>>>(Zs[l], dZ, (long long)rows * no);
            DF_CHECK_LAUNCH();
        }
        const float* in = (l == 0) ? X : As[l - 1];
        // dW = dZ^T in (no x ni); db = colsum dZ; d(in) = dZ W (rows x ni)
        sgemm(m->stream, true, false, no, ni, rows, 1.f, dZ, no, in, ni, 0.f, m->G.p + m->woff[l], ni);
        colsum_kernel<<<nb(no), 256, 0, m->stream>>>(dZ, rows, no, m->G.p + m->boff[l]);
        DF_CHECK_LAUNCH();
        if (l > 0) sgemm(m->stream, false, false, rows, ni, no, 1.f, dZ, no, m->P.p + m->woff[l], ni, 0.f, w.dA[l - 1].p, ni);
    }
    std::vector<float> part(256);
    DF_CUDA(cudaMemcpyAsync(part.data(), w.part.p, 256 * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    DF_CUDA(cudaStreamSynchronize(m->stream));
    double s = 0;
    for (float v : part) s += v;
    return (float)s;
}

// ---------------------------------------------------------------------------------------------
// geometry: water frames, features and rotation matrices for real solid harmonics (l <= 2)
// ---------------------------------------------------------------------------------------------
struct Frame {
    double O[3];
    double R[3][3];   // columns x, y, z of the molecular frame in laboratory coordinates
};

void normalize(double* v) {
    const double r = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int d = 0; d < 3; ++d) v[d] /= r;
}

// waters as consecutive (O, H, H) atoms; z along the H-O-H bisector, x along H1 - H2
std::vector<Frame> water_frames(const df_atom* atoms, int natom) {
    if (natom % 3) throw Error{DF_E_ARG, "learned guess: atoms must be (O, H, H) triples"};
    std::vector<Frame> fr(natom / 3);
    for (int w = 0; w < natom / 3; ++w) {
        const df_atom &o = atoms[3 * w], &h1 = atoms[3 * w + 1], &h2 = atoms[3 * w + 2];
        if (o.Z != 8 || h1.Z != 1 || h2.Z != 1) throw Error{DF_E_ARG, "learned guess: atoms must be (O, H, H) triples"};
        double z[3], x[3], y[3];
        for (int d = 0; d < 3; ++d) {
            z[d] = (h1.xyz[d] - o.xyz[d]) + (h2.xyz[d] - o.xyz[d]);
            x[d] = h1.xyz[d] - h2.xyz[d];
        }
        normalize(z);
        const double dot = x[0] * z[0] + x[1] * z[1] + x[2] * z[2];
        for (int d = 0; d < 3; ++d) x[d] -= dot * z[d];
        normalize(x);
        y[0] = z[1] * x[2] - z[2] * x[1];
        y[1] = z[2] * x[0] - z[0] * x[2];
        y[2] = z[0] * x[1] - z[1] * x[0];
        for (int d = 0; d < 3; ++d) {
            fr[w].O[d] = o.xyz[d];
            fr[w].R[d][0] = x[d];
            fr[w].R[d][1] = y[d];
            fr[w].R[d][2] = z[d];
        }
    }
    return fr;
}

// D^l(Q) with S_lm(Q u) = sum_m' D_mm' S_lm'(u) for the real solid harmonics of cart_sph.cuh:
// l = 1: S = (y, z, x) = P u, so D = P Q P^T. l = 2: S_m(u) = u^T Q_m u with orthogonal traceless Q_m
// (Frobenius norm^2 = 3/2), so D_mm' = <Q^T Q_m Q, Q_m'> / (3/2).
void rotation_l1(const double Q[3][3], double D[3][3]) {
    const int p[3] = {1, 2, 0};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) D[a][b] = Q[p[a]][p[b]];
}

void rotation_l2(const double Q[3][3], double D[5][5]) {
    const double s3 = std::sqrt(3.0);
    double Qm[5][3][3] = {};
    Qm[0][0][1] = Qm[0][1][0] = s3 / 2;     // sqrt3 xy
    Qm[1][1][2] = Qm[1][2][1] = s3 / 2;     // sqrt3 yz
    Qm[2][0][0] = Qm[2][1][1] = -0.5;       // z^2 - (x^2 + y^2)/2
    Qm[2][2][2] = 1.0;
    Qm[3][0][2] = Qm[3][2][0] = s3 / 2;     // sqrt3 xz
    Qm[4][0][0] = s3 / 2;                   // sqrt3/2 (x^2 - y^2)
    Qm[4][1][1] = -s3 / 2;
    for (int a = 0; a < 5; ++a) {
        double T[3][3] = {};   // Q^T Qm_a Q
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) T[i][j] += Q[k][i] * Qm[a][k][l] * Q[l][j];
        for (int b = 0; b < 5; ++b) {
            double s = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) s += T[i][j] * Qm[b][i][j];
            D[a][b] = s / 1.5;
        }
    }
}

// M (nb x nb) for one water's functions: block-diagonal D^l(R^T) per shell; the reference-frame
// function a equals sum_a' M[a][a'] times laboratory function a'
void water_rotation(const df_handle* h, int w, const Frame& f, int nbw, std::vector<double>& M, int& first) {
    double Rt[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Rt[i][j] = f.R[j][i];
    double D1[3][3], D2[5][5];
    rotation_l1(Rt, D1);
    rotation_l2(Rt, D2);
    M.assign((size_t)nbw * nbw, 0.0);
    first = -1;
    int off = 0, local = 0;
    for (const df_shell& s : h->basis) {
        const int ns = 2 * s.l + 1;
        if (s.atom >= 3 * w && s.atom < 3 * w + 3) {
            if (first < 0) first = off;
            if (local + ns > nbw) throw Error{DF_E_ARG, "learned guess: unexpected basis layout"};
            for (int a = 0; a < ns; ++a)
                for (int b = 0; b < ns; ++b)
                    M[(size_t)(local + a) * nbw + local + b] = s.l == 0 ? 1.0 : (s.l == 1 ? D1[a][b] : D2[a][b]);
            local += ns;
        }
        off += ns;
    }
    if (local != nbw) throw Error{DF_E_ARG, "learned guess: every water needs the same basis"};
}

int water_nbf(const df_handle* h) {
    int nbw = 0;
    for (const df_shell& s : h->basis)
        if (s.atom < 3) nbw += 2 * s.l + 1;
    return nbw;
}

// features of water w (DF_MLP_NFEAT values): Gaussian radial histograms of O-O, O-H, H1-O, H2-O
// distances (12 centres 3.5 + 0.9 k bohr, width 0.6 bohr, cutoff 15 bohr) and the coordinates of
// the three nearest other O atoms in the molecule's frame (divided by 10 bohr)
constexpr int NRAD = 12;
constexpr int NFEAT = 4 * NRAD + 9;
void water_features(const df_atom* atoms, int natom, const std::vector<Frame>& fr, int w, float* out) {
    for (int i = 0; i < NFEAT; ++i) out[i] = 0.f;
    auto dist = [&](int a, int b) {
        double r2 = 0;
        for (int d = 0; d < 3; ++d) r2 += (atoms[a].xyz[d] - atoms[b].xyz[d]) * (atoms[a].xyz[d] - atoms[b].xyz[d]);
        return std::sqrt(r2);
    };
    auto hist = [&](float* f, double r) {
        if (r > 15.0) return;
        for (int k = 0; k < NRAD; ++k) {
            const double c = 3.5 + 0.9 * k;
            f[k] += (float)std::exp(-(r - c) * (r - c) / (2 * 0.36));
        }
    };
    std::vector<std::pair<double, int>> near;
    for (int a = 0; a < natom; ++a) {
        if (a / 3 == w) continue;
        if (atoms[a].Z == 8) {
            hist(out, dist(3 * w, a));
            hist(out + 2 * NRAD, dist(3 * w + 1, a));
            hist(out + 3 * NRAD, dist(3 * w + 2, a));
            near.push_back({dist(3 * w, a), a});
        } else {
            hist(out + NRAD, dist(3 * w, a));
        }
    }
    std::sort(near.begin(), near.end());
    for (int q = 0; q < 3 && q < (int)near.size(); ++q) {
        const int a = near[q].second;
        for (int c = 0; c < 3; ++c) {
            double v = 0;
            for (int d = 0; d < 3; ++d) v += fr[w].R[d][c] * (atoms[a].xyz[d] - fr[w].O[d]);
            out[4 * NRAD + 3 * q + c] = (float)(v / 10.0);
        }
    }
}

// pair features of the ordered water pair (w1, w2) (DF_MLP_NPFEAT values): the atoms of w2 in w1's frame
// relative to w1's O (divided by 10 bohr), 5 bohr / r for the nine atom pairs between the two waters, and
// a Gaussian expansion of the O-O distance (8 centres 4.5 + 0.5 k bohr, width 0.35 bohr)
constexpr int NPFEAT = 26;
void pair_features(const df_atom* atoms, const std::vector<Frame>& fr, int w1, int w2, float* out) {
    auto dist = [&](int a, int b) {
        double r2 = 0;
        for (int d = 0; d < 3; ++d) r2 += (atoms[a].xyz[d] - atoms[b].xyz[d]) * (atoms[a].xyz[d] - atoms[b].xyz[d]);
        return std::sqrt(r2);
    };
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            double v = 0;
            for (int d = 0; d < 3; ++d) v += fr[w1].R[d][c] * (atoms[3 * w2 + a].xyz[d] - fr[w1].O[d]);
            out[3 * a + c] = (float)(v / 10.0);
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) out[9 + 3 * a + b] = (float)(5.0 / dist(3 * w1 + a, 3 * w2 + b));
    const double r = dist(3 * w1, 3 * w2);
    for (int k = 0; k < 8; ++k) {
        const double c = 4.5 + 0.5 * k;
        out[18 + k] = (float)std::exp(-(r - c) * (r - c) / (2 * 0.35 * 0.35));
    }
}

// ordered pairs (w1 != w2) with O-O distance <= cutoff, by w1 then w2
std::vector<std::pair<int, int>> water_pair_list(const df_atom* atoms, int natom, double cutoff) {
    std::vector<std::pair<int, int>> out;
    const int nw = natom / 3;
    for (int w1 = 0; w1 < nw; ++w1)
        for (int w2 = 0; w2 < nw; ++w2) {
            if (w1 == w2) continue;
            double r2 = 0;
            for (int d = 0; d < 3; ++d) {
                const double x = atoms[3 * w1].xyz[d] - atoms[3 * w2].xyz[d];
                r2 += x * x;
            }
            if (r2 <= cutoff * cutoff) out.push_back({w1, w2});
        }
    return out;
}

// C = A B (nb x nb, row-major); tA / tB use the transposes
void small_mm(const std::vector<double>& A, bool tA, const std::vector<double>& B, bool tB, int nb,
              std::vector<double>& C) {
    C.assign((size_t)nb * nb, 0.0);
    for (int i = 0; i < nb; ++i)
        for (int k = 0; k < nb; ++k) {
            const double a = tA ? A[(size_t)k * nb + i] : A[(size_t)i * nb + k];
            if (a == 0.0) continue;
            for (int j = 0; j < nb; ++j) C[(size_t)i * nb + j] += a * (tB ? B[(size_t)j * nb + k] : B[(size_t)k * nb + j]);
        }
}

}  // namespace
}  // namespace dfhf

using namespace dfhf;

extern "C" {

int df_mlp_create(int nin, int nhidden, int nlayers, int nout, unsigned long long seed, df_mlp** out) {
    if (!out || nin < 1 || nhidden < 1 || nlayers < 1 || nout < 1) return DF_E_ARG;
    *out = nullptr;
    df_mlp* m = new df_mlp();
    try {
        m->nin = nin;
        m->nh = nhidden;
        m->nlayers = nlayers;
        m->nout = nout;
        m->dims.push_back(nin);
        for (int l = 0; l < nlayers; ++l) m->dims.push_back(nhidden);
        m->dims.push_back(nout);
        long long off = 0;
        for (size_t l = 0; l + 1 < m->dims.size(); ++l) {
            m->woff.push_back(off);
            off += (long long)m->dims[l] * m->dims[l + 1];
            m->boff.push_back(off);
            off += m->dims[l + 1];
        }
        m->nparams = off;
        // He initialisation from a seeded host generator
        std::vector<float> p(off, 0.f);
        std::mt19937_64 gen(seed);
        for (size_t l = 0; l + 1 < m->dims.size(); ++l) {
            std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / m->dims[l]));
            for (long long i = 0; i < (long long)m->dims[l] * m->dims[l + 1]; ++i) p[m->woff[l] + i] = (float)nd(gen);
        }
        DF_CUDA(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking));
        m->P.alloc(off);
        m->G.alloc(off);
        m->Mom.alloc(off);
        m->Vel.alloc(off);
        m->Pbf.alloc(off);
        DF_CUDA(cudaMemcpyAsync(m->P.p, p.data(), off * sizeof(float), cudaMemcpyHostToDevice, m->stream));
        m->Mom.zero(m->stream);
        m->Vel.zero(m->stream);
        DF_CUDA(cudaStreamSynchronize(m->stream));
    } catch (const Error& e) {
        df_mlp_free(m);
        return e.code;
    }
    *out = m;
    return DF_OK;
}

void df_mlp_free(df_mlp* m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    m->P.release();
    m->G.release();
    m->Mom.release();
    m->Vel.release();
    m->Pbf.release();
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

long long df_mlp_nparams(const df_mlp* m) { return m ? m->nparams : DF_E_ARG; }

int df_mlp_params(df_mlp* m, float* host, int set) {
    if (!m || !host) return DF_E_ARG;
    try {
        if (set) {
            DF_CUDA(cudaMemcpyAsync(m->P.p, host, m->nparams * sizeof(float), cudaMemcpyHostToDevice, m->stream));
            m->adam_t = 0;
            m->Mom.zero(m->stream);
            m->Vel.zero(m->stream);
        } else {
            DF_CUDA(cudaMemcpyAsync(host, m->P.p, m->nparams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        }
        DF_CUDA(cudaStreamSynchronize(m->stream));
    } catch (const Error& e) {
        return e.code;
    }
    return DF_OK;
}

int df_mlp_gradients(df_mlp* m, const float* X, const float* Y, int ns, float* grad, float* loss) {
    if (!m || !X || !Y || ns < 1 || !grad) return DF_E_ARG;
    try {
        DevBuf<float> dX, dYt;
        dX.alloc((size_t)ns * m->nin);
        dYt.alloc((size_t)ns * m->nout);
        DF_CUDA(cudaMemcpyAsync(dX.p, X, sizeof(float) * ns * m->nin, cudaMemcpyHostToDevice, m->stream));
        DF_CUDA(cudaMemcpyAsync(dYt.p, Y, sizeof(float) * ns * m->nout, cudaMemcpyHostToDevice, m->stream));
        Work w;
        w.alloc(m, ns);
        const float l = loss_and_grad(m, dX.p, dYt.p, ns, w);
        if (loss) *loss = l;
        DF_CUDA(cudaMemcpyAsync(grad, m->G.p, m->nparams * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        DF_CUDA(cudaStreamSynchronize(m->stream));
        w.release();
        dX.release();
        dYt.release();
    } catch (const Error& e) {
        return e.code;
    }
    return DF_OK;
}

int df_mlp_train(df_mlp* m, const float* X, const float* Y, int ns, int epochs, int batch, float lr,
                 unsigned long long seed, float* loss_history) {
    if (!m || !X || !Y || ns < 1 || epochs < 1 || batch < 1 || !(lr > 0)) return DF_E_ARG;
    try {
        batch = std::min(batch, ns);
        DevBuf<float> dX, dY, bx, by;
        dX.alloc((size_t)ns * m->nin);
        dY.alloc((size_t)ns * m->nout);
        bx.alloc((size_t)batch * m->nin);
        by.alloc((size_t)batch * m->nout);
        DF_CUDA(cudaMemcpyAsync(dX.p, X, sizeof(float) * ns * m->nin, cudaMemcpyHostToDevice, m->stream));
        DF_CUDA(cudaMemcpyAsync(dY.p, Y, sizeof(float) * ns * m->nout, cudaMemcpyHostToDevice, m->stream));
        Work w;
        w.alloc(m, batch);
        std::mt19937_64 gen(seed);
        std::vector<int> perm(ns);
        for (int i = 0; i < ns; ++i) perm[i] = i;
        for (int ep = 0; ep < epochs; ++ep) {
            std::shuffle(perm.begin(), perm.end(), gen);
            double ep_loss = 0;
            int nbatches = 0;
            for (int b0 = 0; b0 + batch <= ns; b0 += batch) {
                for (int r = 0; r < batch; ++r) {
                    const int src = perm[b0 + r];
                    DF_CUDA(cudaMemcpyAsync(bx.p + (long long)r * m->nin, dX.p + (long long)src * m->nin,
                                            sizeof(float) * m->nin, cudaMemcpyDeviceToDevice, m->stream));
                    DF_CUDA(cudaMemcpyAsync(by.p + (long long)r * m->nout, dY.p + (long long)src * m->nout,
                                            sizeof(float) * m->nout, cudaMemcpyDeviceToDevice, m->stream));
                }
                ep_loss += loss_and_grad(m, bx.p, by.p, batch, w);
                ++nbatches;
                ++m->adam_t;
                const float b1 = 0.9f, b2 = 0.999f;
                const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
                adam_kernel<<<nb(m->nparams), 256, 0, m->stream>>>(m->P.p, m->G.p, m->Mom.p, m->Vel.p, m->nparams, lr, b1,
                                                                  b2, 1e-8f, c1, c2);
                DF_CHECK_LAUNCH();
            }
            if (loss_history) loss_history[ep] = (float)(ep_loss / std::max(1, nbatches));
        }
        DF_CUDA(cudaStreamSynchronize(m->stream));
        w.release();
        dX.release();
        dY.release();
        bx.release();
        by.release();
    } catch (const Error& e) {
        return e.code;
    }
    return DF_OK;
}

int df_mlp_predict(df_mlp* m, const float* X, int ns, int bf16, float* Y) {
    if (!m || !X || !Y || ns < 1) return DF_E_ARG;
    try {
        const int L = (int)m->dims.size() - 1;
        DevBuf<float> dX, out;
        dX.alloc((size_t)ns * m->nin);
        out.alloc((size_t)ns * m->nout);
        DF_CUDA(cudaMemcpyAsync(dX.p, X, sizeof(float) * ns * m->nin, cudaMemcpyHostToDevice, m->stream));
        if (!bf16) {
            Work w;
            w.alloc(m, ns);
            std::vector<float*> Zs(L), As(L);
            for (int l = 0; l < L; ++l) {
                Zs[l] = w.Z[l].p;
                As[l] = w.A[l].p;
            }
            forward(m, dX.p, ns, Zs, As);
            DF_CUDA(cudaMemcpyAsync(Y, As[L - 1], sizeof(float) * ns * m->nout, cudaMemcpyDeviceToHost, m->stream));
            DF_CUDA(cudaStreamSynchronize(m->stream));
            w.release();
        } else {
            to_bf16_kernel<<<nb(m->nparams), 256, 0, m->stream>>>(m->P.p, m->nparams, m->Pbf.p);
            DF_CHECK_LAUNCH();
            int maxw = m->nin;
            for (int d : m->dims) maxw = std::max(maxw, d);
            DevBuf<__nv_bfloat16> a, b;
            a.alloc((size_t)ns * maxw);
            b.alloc((size_t)ns * maxw);
            to_bf16_kernel<<<nb((long long)ns * m->nin), 256, 0, m->stream>>>(dX.p, (long long)ns * m->nin, a.p);
            DF_CHECK_LAUNCH();
            for (int l = 0; l < L; ++l) {
                const int ni = m->dims[l], no = m->dims[l + 1];
                const bool last = l == L - 1;
                bf16_layer_kernel<<<nb((long long)ns * no * 32), 256, 0, m->stream>>>(
                    a.p, ns, ni, m->Pbf.p + m->woff[l], m->Pbf.p + m->boff[l], no, !last, last ? nullptr : b.p,
                    last ? out.p : nullptr);
                DF_CHECK_LAUNCH();
                std::swap(a, b);
            }
            DF_CUDA(cudaMemcpyAsync(Y, out.p, sizeof(float) * ns * m->nout, cudaMemcpyDeviceToHost, m->stream));
            DF_CUDA(cudaStreamSynchronize(m->stream));
            a.release();
            b.release();
        }
        dX.release();
        out.release();
    } catch (const Error& e) {
        return e.code;
    }
    return DF_OK;
}

int df_water_features(const df_atom* atoms, int natom, float* out) {
    if (!atoms || natom < 3 || !out) return DF_E_ARG;
    try {
        const std::vector<Frame> fr = water_frames(atoms, natom);
        for (int w = 0; w < natom / 3; ++w) water_features(atoms, natom, fr, w, out + (size_t)w * NFEAT);
    } catch (const Error& e) {
        return e.code;
    }
    return NFEAT;
}

// reference-frame diagonal blocks of D (host, n x n): out[w] = upper triangle of M D_w M^T
int df_water_blocks(df_handle* h, const double* D, float* out) {
    if (!h || !D || !out) return DF_E_ARG;
    try {
        const std::vector<Frame> fr = water_frames(h->atoms.data(), (int)h->atoms.size());
        const int nbw = water_nbf(h);
        std::vector<double> M, T((size_t)nbw * nbw);
        const int ntri = nbw * (nbw + 1) / 2;
        for (int w = 0; w < (int)fr.size(); ++w) {
            int first = 0;
            water_rotation(h, w, fr[w], nbw, M, first);
            // T = M Dw M^T
            std::vector<double> MD((size_t)nbw * nbw, 0.0);
            for (int a = 0; a < nbw; ++a)
                for (int c = 0; c < nbw; ++c) {
                    const double mac = M[(size_t)a * nbw + c];
                    if (mac == 0.0) continue;
                    for (int b = 0; b < nbw; ++b) MD[(size_t)a * nbw + b] += mac * D[(size_t)(first + c) * h->n + first + b];
                }
            for (int a = 0; a < nbw; ++a)
                for (int b = 0; b < nbw; ++b) {
                    double s = 0;
                    for (int c = 0; c < nbw; ++c) s += MD[(size_t)a * nbw + c] * M[(size_t)b * nbw + c];
                    T[(size_t)a * nbw + b] = s;
                }
            int k = 0;
            for (int a = 0; a < nbw; ++a)
                for (int b = a; b < nbw; ++b) out[(size_t)w * ntri + k++] = (float)T[(size_t)a * nbw + b];
        }
    } catch (const Error& e) {
        return fail_code(h, e);
    }
    return DF_OK;
}

// learned D0 for a water cluster: features -> MLP (BF16 inference if bf16) -> blocks -> D0 (host)
int df_mlp_guess(df_handle* h, df_mlp* m, int bf16, double* D0) {
    if (!h || !m || !D0) return DF_E_ARG;
    const int natom = (int)h->atoms.size();
    if (natom % 3) return DF_E_ARG;
    const int nw = natom / 3;
    const int nbw = water_nbf(h);
    if (m->nin != NFEAT || m->nout != nbw * (nbw + 1) / 2) {
        h->last_error = "df_mlp_guess: network shape does not match the features / water basis";
        return DF_E_ARG;
    }
    std::vector<float> X((size_t)nw * NFEAT), Y((size_t)nw * m->nout);
    int rc = df_water_features(h->atoms.data(), natom, X.data());
    if (rc < 0) return rc;
    rc = df_mlp_predict(m, X.data(), nw, bf16, Y.data());
    if (rc != DF_OK) return rc;
    return df_water_density(h, Y.data(), D0);
}

int df_water_pairs(const df_atom* atoms, int natom, double cutoff, int* pairs, int max_pairs, float* feats) {
    if (!atoms || natom < 3 || !(cutoff > 0) || max_pairs < 0 || (max_pairs > 0 && !pairs)) return DF_E_ARG;
    try {
        const std::vector<Frame> fr = water_frames(atoms, natom);
        const auto list = water_pair_list(atoms, natom, cutoff);
        for (int k = 0; k < (int)list.size() && k < max_pairs; ++k) {
            pairs[2 * k] = list[k].first;
            pairs[2 * k + 1] = list[k].second;
            if (feats) pair_features(atoms, fr, list[k].first, list[k].second, feats + (size_t)k * NPFEAT);
        }
        return (int)list.size();
    } catch (const Error& e) {
        return e.code;
    }
}

// out[k] = M_1 D[w1][w2] M_2^T (nb x nb, row-major): the block of the ordered pair in w1's frame (M_2 rotates
// w2's functions by w1's frame)
int df_pair_blocks(df_handle* h, const double* D, const int* pairs, int npairs, float* out) {
    if (!h || !D || npairs < 0 || (npairs > 0 && (!pairs || !out))) return DF_E_ARG;
    try {
        const std::vector<Frame> fr = water_frames(h->atoms.data(), (int)h->atoms.size());
        const int nbw = water_nbf(h), nw = (int)fr.size();
        std::vector<double> M1, M2, Dl((size_t)nbw * nbw), T1, T;
        for (int k = 0; k < npairs; ++k) {
            const int w1 = pairs[2 * k], w2 = pairs[2 * k + 1];
            if (w1 < 0 || w2 < 0 || w1 >= nw || w2 >= nw || w1 == w2) throw Error{DF_E_ARG, "df_pair_blocks: bad pair"};
            int f1 = 0, f2 = 0;
            water_rotation(h, w1, fr[w1], nbw, M1, f1);
            water_rotation(h, w2, fr[w1], nbw, M2, f2);
            for (int a = 0; a < nbw; ++a)
                for (int b = 0; b < nbw; ++b) Dl[(size_t)a * nbw + b] = D[(size_t)(f1 + a) * h->n + f2 + b];
            small_mm(M1, false, Dl, false, nbw, T1);
            small_mm(T1, false, M2, true, nbw, T);
            for (size_t i = 0; i < T.size(); ++i) out[(size_t)k * nbw * nbw + i] = (float)T[i];
        }
    } catch (const Error& e) {
        return fail_code(h, e);
    }
    return DF_OK;
}

// D0 += the laboratory-frame pair blocks M_1^T T M_2 at [w1][w2] and their transposes at [w2][w1]; a pair
// listed in both orders contributes the mean of its two blocks
int df_pair_density(df_handle* h, const float* blocks, const int* pairs, int npairs, double* D0) {
    if (!h || !D0 || npairs < 0 || (npairs > 0 && (!pairs || !blocks))) return DF_E_ARG;
    try {
        const std::vector<Frame> fr = water_frames(h->atoms.data(), (int)h->atoms.size());
        const int nbw = water_nbf(h), nw = (int)fr.size();
        std::vector<int> count((size_t)nw * nw, 0);
        for (int k = 0; k < npairs; ++k) {
            const int w1 = pairs[2 * k], w2 = pairs[2 * k + 1];
            if (w1 < 0 || w2 < 0 || w1 >= nw || w2 >= nw || w1 == w2) throw Error{DF_E_ARG, "df_pair_density: bad pair"};
            ++count[(size_t)std::min(w1, w2) * nw + std::max(w1, w2)];
        }
        std::vector<double> M1, M2, T((size_t)nbw * nbw), T1, L;
        for (int k = 0; k < npairs; ++k) {
            const int w1 = pairs[2 * k], w2 = pairs[2 * k + 1];
            const double wgt = 1.0 / count[(size_t)std::min(w1, w2) * nw + std::max(w1, w2)];
            int f1 = 0, f2 = 0;
            water_rotation(h, w1, fr[w1], nbw, M1, f1);
            water_rotation(h, w2, fr[w1], nbw, M2, f2);
            for (size_t i = 0; i < T.size(); ++i) T[i] = blocks[(size_t)k * nbw * nbw + i];
            small_mm(M1, true, T, false, nbw, T1);
            small_mm(T1, false, M2, false, nbw, L);
            for (int a = 0; a < nbw; ++a)
                for (int b = 0; b < nbw; ++b) {
                    const double v = wgt * L[(size_t)a * nbw + b];
                    D0[(size_t)(f1 + a) * h->n + f2 + b] += v;
                    D0[(size_t)(f2 + b) * h->n + f1 + a] += v;
                }
        }
    } catch (const Error& e) {
        return fail_code(h, e);
    }
    return DF_OK;
}

// learned D0 with pair blocks: the diagonal blocks from m (df_mlp_guess) plus the blocks of every water pair
// within `cutoff` bohr (O-O) from mp, in both orders
int df_mlp_guess_pairs(df_handle* h, df_mlp* m, df_mlp* mp, double cutoff, int bf16, double* D0) {
    if (!h || !m || !mp || !D0 || !(cutoff > 0)) return DF_E_ARG;
    const int nbw = water_nbf(h);
    if (mp->nin != NPFEAT || mp->nout != nbw * nbw) {
        h->last_error = "df_mlp_guess_pairs: pair network shape does not match the pair features / water basis";
        return DF_E_ARG;
    }
    int rc = df_mlp_guess(h, m, bf16, D0);
    if (rc != DF_OK) return rc;
    const int natom = (int)h->atoms.size();
    const int np = df_water_pairs(h->atoms.data(), natom, cutoff, nullptr, 0, nullptr);
    if (np < 0) return np;
    if (np == 0) return DF_OK;
    std::vector<int> pairs(2 * (size_t)np);
    std::vector<float> X((size_t)np * NPFEAT), Y((size_t)np * mp->nout);
    rc = df_water_pairs(h->atoms.data(), natom, cutoff, pairs.data(), np, X.data());
    if (rc < 0) return rc;
    rc = df_mlp_predict(mp, X.data(), np, bf16, Y.data());
    if (rc != DF_OK) return rc;
    return df_pair_density(h, Y.data(), pairs.data(), np, D0);
}

// D0 (host n x n) from reference-frame blocks (nwater x ntri): block-diagonal M^T T_w M
int df_water_density(df_handle* h, const float* blocks, double* D0) {
    if (!h || !blocks || !D0) return DF_E_ARG;
    try {
        const std::vector<Frame> fr = water_frames(h->atoms.data(), (int)h->atoms.size());
        const int nbw = water_nbf(h);
        const int ntri = nbw * (nbw + 1) / 2;
        std::fill(D0, D0 + (size_t)h->n * h->n, 0.0);
        std::vector<double> M, T((size_t)nbw * nbw), TM((size_t)nbw * nbw);
        for (int w = 0; w < (int)fr.size(); ++w) {
            int first = 0;
            water_rotation(h, w, fr[w], nbw, M, first);
            int k = 0;
            for (int a = 0; a < nbw; ++a)
                for (int b = a; b < nbw; ++b) T[(size_t)a * nbw + b] = T[(size_t)b * nbw + a] = blocks[(size_t)w * ntri + k++];
            std::fill(TM.begin(), TM.end(), 0.0);
            for (int a = 0; a < nbw; ++a)
                for (int c = 0; c < nbw; ++c) {
                    const double t = T[(size_t)a * nbw + c];
                    for (int b = 0; b < nbw; ++b) TM[(size_t)a * nbw + b] += t * M[(size_t)c * nbw + b];
                }
            for (int a = 0; a < nbw; ++a)
                for (int b = 0; b < nbw; ++b) {
                    double s = 0;
                    for (int c = 0; c < nbw; ++c) s += M[(size_t)c * nbw + a] * TM[(size_t)c * nbw + b];
                    D0[(size_t)(first + a) * h->n + first + b] = s;
                }
        }
    } catch (const Error& e) {
        return fail_code(h, e);
    }
    return DF_OK;
}

}  // extern "C"
