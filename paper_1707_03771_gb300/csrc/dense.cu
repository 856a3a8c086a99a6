// FP64 dense contractions on the CUDA cores (DFMA).
//
// On GB300 the FP64 pipe delivers about 1 TFLOP/s (DFMA and DMMA alike), so these kernels are
// bound by FP64 issue, not by memory: a 64x64 register-blocked tile with 4x4 outputs per thread and
// operands staged through shared memory keeps the pipe busy with ample reuse.
//   - dgemm: general row-major C = alpha op(A) op(B) + beta C (SCF algebra).
//   - dtrmm_lower: C = L A for lower-triangular L (metric whitening B = L^-1 (Q|mu nu), paper eq. 1,
//     third form); block rows skip the zero upper triangle.
//   - whiten_fp64_inplace: A <- L A for lower-triangular L, in place, one 64-row block of L per launch
//     from the last block up (the FP64 whitening).
//   - y_transform: Y_{P,mu i} = sum_nu B_{P,mu nu} C_{nu i} reading the packed symmetric B
//     (paper eq. 1, first form); each stored off-diagonal tile serves both (I,J) and (J,I).
//   - k_syrk: K_{mu nu} = sum_{P,i} Y_{P,mu i} Y_{P,nu i} over lower tile pairs with split-K partial
//     sums (paper eq. 2, first form), reduced deterministically.
#include "common.cuh"

namespace dfhf {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;
constexpr int NTHR = 256;   // 16 x 16 threads, 4 x 4 outputs each

// accumulate one BK slice: As[k][m], Bs[k][n]
__device__ __forceinline__ void mma_tile(const double (*As)[BM + 1], const double (*Bs)[BN + 1], int tx, int ty,
                                         double acc[4][4]) {
#pragma unroll
    for (int k = 0; k < BK; ++k) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
}

__global__ void __launch_bounds__(NTHR) dgemm_kernel(bool ta, bool tb, int m, int n, int k, double alpha,
                                                     const double* __restrict__ A, long long lda,
                                                     const double* __restrict__ B, long long ldb, double beta,
                                                     double* __restrict__ C, long long ldc, bool lower_a) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * BM;
    const long long n0 = (long long)blockIdx.x * BN;
    double acc[4][4] = {};
    const int kend = lower_a ? min(k, m0 + BM) : k;
    for (int k0 = 0; k0 < kend; k0 += BK) {
        for (int idx = tid; idx < BM * BK; idx += NTHR) {
            int r, c;
            if (!ta) { r = idx / BK; c = idx % BK; }
            else { c = idx / BM; r = idx % BM; }
            const int gm = m0 + r, gk = k0 + c;
            double v = 0.0;
            if (gm < m && gk < k) v = ta ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
            As[c][r] = v;
        }
        for (int idx = tid; idx < BK * BN; idx += NTHR) {
            int r, c;
            if (!tb) { r = idx / BN; c = idx % BN; }
            else { c = idx / BK; r = idx % BK; }
            const int gk = k0 + r;
            const long long gn = n0 + c;
            double v = 0.0;
            if (gk < k && gn < n) v = tb ? B[gn * ldb + gk] : B[(long long)gk * ldb + gn];
            Bs[r][c] = v;
        }
        __syncthreads();
        mma_tile(As, Bs, tx, ty, acc);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + ty + 16 * i;
        if (gm >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long gn = n0 + tx + 16 * j;
            if (gn >= n) continue;
            double* c = C + (long long)gm * ldc + gn;
            *c = alpha * acc[i][j] + (beta == 0.0 ? 0.0 : beta * *c);
        }
    }
}

// Y[P][mu][i] (rows padded to np, columns to ldy) from packed B row P and Cpad[np][ldy]
__global__ void __launch_bounds__(NTHR) y_transform_kernel(const double* __restrict__ B, long long row, int nt,
                                                           const double* __restrict__ Cp, int ldy, int ncol,
                                                           double* __restrict__ Y) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int I = blockIdx.y;
    const int i0 = blockIdx.x * BN;
    const long long P = blockIdx.z;
    const double* Brow = B + P * row;
    double acc[4][4] = {};
    for (int J = 0; J < nt; ++J) {
        const bool direct = J <= I;
        const double* tile = Brow + (direct ? tile_pair(I, J) : tile_pair(J, I)) * (TS * TS);
        for (int k0 = 0; k0 < TS; k0 += BK) {
            // A operand: element (mu_local r, nu_local c) of B_P
            for (int idx = tid; idx < BM * BK; idx += NTHR) {
                int r, c;
                if (direct) { r = idx / BK; c = idx % BK; }
                else { c = idx / BM; r = idx % BM; }
                As[c][r] = direct ? tile[r * TS + k0 + c] : tile[(k0 + c) * TS + r];
            }
            for (int idx = tid; idx < BK * BN; idx += NTHR) {
                const int r = idx / BN, c = idx % BN;
                const int gi = i0 + c;
                Bs[r][c] = (gi < ncol) ? Cp[(long long)(J * TS + k0 + r) * ldy + gi] : 0.0;
            }
            __syncthreads();
            mma_tile(As, Bs, tx, ty, acc);
            __syncthreads();
        }
    }
    double* Yp = Y + P * (long long)nt * TS * ldy;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int mu = I * TS + ty + 16 * i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gi = i0 + tx + 16 * j;
            if (gi < ldy) Yp[(long long)mu * ldy + gi] = (gi < ncol) ? acc[i][j] : 0.0;
        }
    }
}

// partial K over auxiliary range of split s for tile pair (I >= J) given by blockIdx.x
__global__ void __launch_bounds__(NTHR) k_syrk_kernel(const double* __restrict__ Y, int naux, int np, int ldy,
                                                      int ncol, int nsplit, const int2* __restrict__ tiles,
                                                      double* __restrict__ Kpart) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int2 IJ = tiles[blockIdx.x];
    const int s = blockIdx.y;
    const int p0 = (int)((long long)naux * s / nsplit), p1 = (int)((long long)naux * (s + 1) / nsplit);
    double acc[4][4] = {};
    for (int P = p0; P < p1; ++P) {
        const double* Yp = Y + (long long)P * np * ldy;
        for (int k0 = 0; k0 < ncol; k0 += BK) {
            for (int idx = tid; idx < BM * BK; idx += NTHR) {
                const int r = idx / BK, c = idx % BK;
                const int gk = k0 + c;
                As[c][r] = (gk < ncol) ? Yp[(long long)(IJ.x * TS + r) * ldy + gk] : 0.0;
                Bs[c][r] = (gk < ncol) ? Yp[(long long)(IJ.y * TS + r) * ldy + gk] : 0.0;
            }
            __syncthreads();
            mma_tile(As, Bs, tx, ty, acc);
            __syncthreads();
        }
    }
    double* Kp = Kpart + (long long)s * np * np;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            Kp[(long long)(IJ.x * TS + ty + 16 * i) * np + IJ.y * TS + tx + 16 * j] = acc[i][j];
}

// K[mu][nu] (n x n) = sum_s Kpart over the stored lower tiles, mirrored
__global__ void k_reduce_kernel(const double* __restrict__ Kpart, int nsplit, int np, int n, double* __restrict__ K) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int mu = (int)(idx / n), nu = (int)(idx % n);
    int a = mu, b = nu;
    if (mu / TS < nu / TS) { a = nu; b = mu; }
    double s = 0.0;
    for (int t = 0; t < nsplit; ++t) s += Kpart[(long long)t * np * np + (long long)a * np + b];
    K[idx] = s;
}

}  // namespace

void dgemm(cudaStream_t s, bool ta, bool tb, int m, int n, int k, double alpha, const double* A, int lda,
           const double* B, int ldb, double beta, double* C, int ldc) {
    dim3 grid((n + BN - 1) / BN, (m + BM - 1) / BM);
    dgemm_kernel<<<grid, NTHR, 0, s>>>(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, false);
    DF_CHECK_LAUNCH();
}

void dtrmm_lower(cudaStream_t s, int m, long long ncol, const double* L, const double* A, double* C, long long ld) {
    const long long chunk = 65535LL * BN;   // grid.x limit
    for (long long c0 = 0; c0 < ncol; c0 += chunk) {
        const long long nc = (ncol - c0 < chunk) ? ncol - c0 : chunk;
        dim3 grid((unsigned)((nc + BN - 1) / BN), (m + BM - 1) / BM);
        dgemm_kernel<<<grid, NTHR, 0, s>>>(false, false, m, (int)nc, m, 1.0, L, m, A + c0, ld, 0.0, C + c0, ld, true);
        DF_CHECK_LAUNCH();
    }
}

// A <- L A in place for lower-triangular L (m x m, row-major) and A (m x ncol, row stride ld). Row block I
// of the result needs rows 0 .. end of block I of A; launching the blocks from the last one up leaves those
// rows unmodified until their own launch. Within a launch a CTA reads only its own column tile and writes it
// after its last read, so no CTA sees another's output.
void whiten_fp64_inplace(cudaStream_t s, int m, long long ncol, const double* L, double* A, long long ld) {
    const long long chunk = 65535LL * BN;   // grid.x limit
    for (int r0 = ((m - 1) / BM) * BM; r0 >= 0; r0 -= BM) {
        const int rows = m - r0 < BM ? m - r0 : BM;
        const int kk = r0 + rows;   // L is zero beyond the diagonal block
        for (long long c0 = 0; c0 < ncol; c0 += chunk) {
            const long long nc = (ncol - c0 < chunk) ? ncol - c0 : chunk;
            dim3 grid((unsigned)((nc + BN - 1) / BN), 1);
            dgemm_kernel<<<grid, NTHR, 0, s>>>(false, false, rows, (int)nc, kk, 1.0, L + (long long)r0 * m, m, A + c0,
                                               ld, 0.0, A + (long long)r0 * ld + c0, ld, false);
            DF_CHECK_LAUNCH();
        }
    }
}

void y_transform_fp64(cudaStream_t s, const double* B, long long row, int nt, int naux, const double* Cp, int ldy,
                      int ncol, double* Y) {
    dim3 grid((ldy + BN - 1) / BN, nt, naux);
    y_transform_kernel<<<grid, NTHR, 0, s>>>(B, row, nt, Cp, ldy, ncol, Y);
    DF_CHECK_LAUNCH();
}

void k_syrk_fp64(cudaStream_t s, const double* Y, int naux, int np, int ldy, int ncol, int nsplit,
                 const int2* tiles, int ntiles, double* Kpart, int n, double* K) {
    dim3 grid(ntiles, nsplit);
    k_syrk_kernel<<<grid, NTHR, 0, s>>>(Y, naux, np, ldy, ncol, nsplit, tiles, Kpart);
    DF_CHECK_LAUNCH();
    const long long tot = (long long)n * n;
    k_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Kpart, nsplit, np, n, K);
    DF_CHECK_LAUNCH();
}

}  // namespace dfhf
