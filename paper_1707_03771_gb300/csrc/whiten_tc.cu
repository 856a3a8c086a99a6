// Metric whitening B = L^-1 (Q|mu nu) (paper eq. 1, third form, with M' = L^-1) on the tcgen05 tensor
// cores by Ozaki splitting.
//
// GB300's FP64 rate is ~1 TFLOP/s; the whitening is naux^2 npair / 2 multiply-adds (24.6 TFLOP at 32
// waters). Each row of L^-1 is scaled by its power of two and written as 7 BF16 digit slices, each pair
// column of the three-index tensor likewise (with its own power of two, transposed so the auxiliary
// index is contiguous); the 28 slice pairs with s + t <= 8 are multiplied on the tensor cores in exact
// FP32 chunks and summed in float-float (ozaki_tc_kernel, whitening mode). With 7 slices the result
// differs from an FP64 product L^-1 A by ~3e-10 of max|B| on the 8-water cluster, well inside the
// ~kappa(L) eps |B| by which two correct FP64 whitenings differ (8e-9 there).
//
// The pair columns are processed in chunks whose transposed slices fit a bounded buffer; when the
// unwhitened tensor is not kept, each chunk's result overwrites the chunk's own columns in place.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>

#include "common.cuh"
#include "ozaki.cuh"

namespace dfhf {

void whiten_tc(cudaStream_t s, int N, const __nv_bfloat16* Ls, const int* eL, const __nv_bfloat16* At, const int* eA,
               int naux, int kp, int ncols, double* out, long long ldo, int* err);

namespace {

typedef __nv_bfloat16 bf16;
constexpr int WS = 7;   // slices

// Output tile width of the whitening kernel (64, or 32 with two CTAs per SM), chosen per size bucket
// (naux / 512) by timing the first two column chunks of the first whitening in that bucket with one
// width each: the candidates run on real work, so the choice costs nothing extra.
std::mutex g_wmu;
std::map<int, int> g_wtile;

// L^-1 (naux x naux, row-major, lower) -> Ls[s][P][Q] (kp columns, zero beyond naux), eL[P]
__global__ void __launch_bounds__(256) slice_rows_kernel(const double* __restrict__ L, int naux, int kp,
                                                         bf16* __restrict__ Ls, long long sstr, int* __restrict__ eL) {
    const int P = blockIdx.x;
    const double* row = L + (long long)P * naux;
    double mx = 0.0;
    for (int q = threadIdx.x; q < naux; q += blockDim.x) mx = fmax(mx, fabs(row[q]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);   // |row| * 2^-e < 1
    if (threadIdx.x == 0) eL[P] = e;
    bf16* o = Ls + (long long)P * kp;
    for (int q = threadIdx.x; q < kp; q += blockDim.x) split_pow2<WS>(q < naux ? row[q] : 0.0, e, o + q, sstr);
}

// eA[c] = exponent of max_Q |A[Q][c0 + c]| for the chunk's columns
__global__ void __launch_bounds__(256) col_exponent_kernel(const double* __restrict__ A, long long ld, int naux,
                                                           long long c0, int nc, int* __restrict__ eA) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const double* a = A + c0 + c;
    double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
    int q = 0;
    for (; q + 4 <= naux; q += 4) {
        m0 = fmax(m0, fabs(a[(long long)q * ld]));
        m1 = fmax(m1, fabs(a[(long long)(q + 1) * ld]));
        m2 = fmax(m2, fabs(a[(long long)(q + 2) * ld]));
        m3 = fmax(m3, fabs(a[(long long)(q + 3) * ld]));
    }
    for (; q < naux; ++q) m0 = fmax(m0, fabs(a[(long long)q * ld]));
    const double mx = fmax(fmax(m0, m1), fmax(m2, m3));
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    eA[c] = e;
}

// At[s][c][Q] (kp per column, zero beyond naux) = slices of A[Q][c0 + c] 2^-eA[c]; 64 x 64 tiles
// transposed through shared memory (reads coalesced along c, writes along Q)
__global__ void __launch_bounds__(256) slice_cols_kernel(const double* __restrict__ A, long long ld, int naux, int kp,
                                                         long long c0, const int* __restrict__ eA,
                                                         bf16* __restrict__ At, long long sstr) {
    __shared__ double tile[64][65];
    const int cb = blockIdx.x * 64, q0 = blockIdx.y * 64;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;   // 64 x 4
    for (int r = ty; r < 64; r += 4) {
        const int q = q0 + r;
        tile[r][tx] = q < naux ? A[(long long)q * ld + c0 + cb + tx] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 64; r += 4) {   // r: column within the tile, tx: Q within the tile
        const int c = cb + r;
        split_pow2<WS>(tile[tx][r], eA[c], At + (long long)c * kp + q0 + tx, sstr);
    }
}

}  // namespace

// B = L^-1 A for the packed tensor A (naux rows of `ncol` doubles, stride ld). `B` may equal `A`
// (in place, chunk by chunk). Scratch: the slices of L^-1 and one chunk of transposed slices.
void whiten_ozaki(cudaStream_t s, int naux, long long ncol, long long ld, const double* Linv, const double* A,
                  double* B) {
    if (ncol % 64) throw Error{DF_E_ARG, "internal: whitening columns not a multiple of 64"};
    const int kp = (naux + 63) / 64 * 64;
    size_t free_b = 0, total_b = 0;
    DF_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const double col_bytes = (double)WS * kp * 2 + 4;
    // the chunk's transposed slices: at most 8 GB (several molecules may whiten at once)
    const double chunk_bytes = std::min(0.4 * (double)free_b, 8.0e9);
    long long nc = (long long)std::min<double>((double)ncol, chunk_bytes / col_bytes);
    nc = std::min<long long>(nc, 1LL << 19) / 4096 * 4096;
    if (nc < 64) nc = std::min<long long>(ncol, 64);
    if (nc > ncol) nc = ncol;
    DevBuf<bf16> Ls, At;
    DevBuf<int> eL, eA, err;
    Ls.alloc((size_t)WS * naux * kp);
    eL.alloc(naux);
    At.alloc((size_t)WS * nc * kp);
    eA.alloc(nc);
    err.alloc(1);
    err.zero(s);
    try {
    slice_rows_kernel<<<naux, 256, 0, s>>>(Linv, naux, kp, Ls.p, (long long)naux * kp, eL.p);
    DF_CHECK_LAUNCH();
    const int bucket = (naux + 511) / 512;
    int tile = 0;
    {
        std::lock_guard<std::mutex> lock(g_wmu);
        auto it = g_wtile.find(bucket);
        if (it != g_wtile.end()) tile = it->second;
    }
    if (const char* f = std::getenv("DFHF_WHITEN_TILE")) {   // fixes the width (tests compare the two)
        const int t = std::atoi(f);
        if (t == 32 || t == 64) tile = t;
    }
    const bool tune = tile == 0 && ncol >= 2 * nc;   // two full-width chunks to compare
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (tune)
        for (auto& e : ev) DF_CUDA(cudaEventCreate(&e));
    int k = 0;
    for (long long c0 = 0; c0 < ncol; c0 += nc, ++k) {
        const int w = (int)std::min<long long>(nc, ncol - c0);
        col_exponent_kernel<<<(w + 255) / 256, 256, 0, s>>>(A, ld, naux, c0, w, eA.p);
        DF_CHECK_LAUNCH();
        slice_cols_kernel<<<dim3(w / 64, kp / 64), 256, 0, s>>>(A, ld, naux, kp, c0, eA.p, At.p, (long long)w * kp);
        DF_CHECK_LAUNCH();
        int use = tile ? tile : 64;
        if (tune && k < 2) {
            use = k == 0 ? 64 : 32;
            DF_CUDA(cudaEventRecord(ev[2 * k], s));
        }
        whiten_tc(s, use, Ls.p, eL.p, At.p, eA.p, naux, kp, w, B + c0, ld, err.p);
        if (tune && k < 2) DF_CUDA(cudaEventRecord(ev[2 * k + 1], s));
        if (tune && k == 1) {
            DF_CUDA(cudaEventSynchronize(ev[3]));
            tile = elapsed_ms(ev[2], ev[3]) < elapsed_ms(ev[0], ev[1]) ? 32 : 64;
            std::lock_guard<std::mutex> lock(g_wmu);
            g_wtile[bucket] = tile;
        }
    }
    if (tune)
        for (auto& e : ev) cudaEventDestroy(e);
    int herr = 0;
    DF_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    DF_CUDA(cudaStreamSynchronize(s));
    if (herr) throw Error{DF_E_TIMEOUT, "tensor-core whitening kernel timed out waiting on a barrier"};
    } catch (...) {
        cudaStreamSynchronize(s);   // queued kernels finish before the scratch buffers are released
        throw;
    }
}

}  // namespace dfhf
