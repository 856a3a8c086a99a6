// Split-precision exchange: K = sum_P Y_P Y_P^T with Y_P = B_P C_occ (paper eq. 1 first form and
// eq. 2 first form) on the BF16 tensor cores, with FP64 accuracy recovered by error-free splitting
// (Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 95 (2012)).
//
// Splitting. A vector x sharing one power-of-two scale 2^e (max|x| < 2^e) is written exactly as
//   x = 2^e sum_{s=1..S} m_s 2^{-7 s} + r,   m_1 in [-128, 128], m_s in [-64, 64] (s > 1),
// with integers m_s (exact in BF16) and |r| <= 2^{e - 7 S - 1}. Scales: per row (P, mu) of B over nu,
// per column i of C over nu, per (mu, block of auxiliary rows) of Y over (P, i).
// Products. sum_k m_s(a_k) m_t(b_k) over a chunk of at most 512 terms is an integer below 2^24 even
// when all pairs with s + t = L are summed into one accumulator (at most 2^14 + 3 * 2^13 per term for
// S <= 5), so the FP32 tensor-core sums are exact whatever the hardware's rounding. Pairs with s + t <= S + 1 are kept (the dropped pairs are
// below 2^{-7(S+1)} relative). After each chunk the integer sums are scaled by the exact power of
// two 2^{e_a + e_b - 7 L} and added into float-float accumulators (hi, lo) with Knuth's TwoSum.
// Y leaves its kernel as (hi, lo) pairs and is re-split with one exponent per (mu, block of the contraction
// over (P, i)): for the tensor-core contraction over the contiguous index k = P ldy + i in blocks of one
// exact chunk, for the mma.sync contraction in blocks of whole auxiliary rows. K leaves as (hi, lo) partial
// sums that are combined in FP64.
// MMA: mma.sync m16n8k16 BF16 -> FP32 (warp-level), operands staged in shared memory by cp.async.
#include <cuda_bf16.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "ozaki.cuh"

namespace dfhf {

namespace {

typedef __nv_bfloat16 bf16;

constexpr int KT = 32;             // contraction tile (elements)
constexpr int LDS = KT + 8;        // padded shared-memory row (bf16): 80 B, conflict-free ldmatrix
constexpr int CHUNK_TILES = 16;    // exchange chunks: whole auxiliary rows, at most 512 elements (exact for S <= 5)
constexpr int SMAX = 5;

// exact 2^e as a float; 0 below the normal range (such contributions are below 2^-126 of the scale)
__device__ __forceinline__ float pow2f(int e) { return e < -126 ? 0.f : __int_as_float((127 + min(e, 127)) << 23); }

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (v - bb);
    hi = s;
    lo += err;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(unsigned* r, const bf16* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float* d, const unsigned* a, const unsigned* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ------------------------------------------------------------------------------------------------
// split of B: packed FP64 tiles -> Bs[s][P][mu][nu] (np x np per P), exponent per (P, mu)
// ------------------------------------------------------------------------------------------------
// tile pair index -> (I, J), I >= J
__device__ __forceinline__ void tile_of(long long tp, int& I, int& J) {
    I = (int)((sqrt(8.0 * (double)tp + 1.0) - 1.0) * 0.5);
    while ((long long)(I + 1) * (I + 2) / 2 <= tp) ++I;
    while ((long long)I * (I + 1) / 2 > tp) --I;
    J = (int)(tp - (long long)I * (I + 1) / 2);
}

// rmax[P][mu] = max_nu |B_P[mu][nu]| as the bit pattern of a non-negative double (ordered like the
// value), gathered tile by tile: rows of tile (I, J) for mu in I, its columns for mu in J (I > J)
__global__ void __launch_bounds__(256) row_max_tiles_kernel(const double* __restrict__ B, long long row, int np,
                                                            unsigned long long* __restrict__ rmax) {
    __shared__ double tile[64][65];
    const long long tp = blockIdx.x, P = blockIdx.y;
    int I, J;
    tile_of(tp, I, J);
    const double* src = B + P * row + tp * 4096;
    for (int i = threadIdx.x; i < 4096; i += 256) tile[i >> 6][i & 63] = fabs(src[i]);
    __syncthreads();
    const int k = threadIdx.x >> 2, q = threadIdx.x & 3;   // row (or column) k, quarter q
    double mr = 0.0, mc = 0.0;
#pragma unroll 4
    for (int j = q * 16; j < q * 16 + 16; ++j) {
        mr = fmax(mr, tile[k][j]);
        mc = fmax(mc, tile[j][k]);
    }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
        mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
        mc = fmax(mc, __shfl_xor_sync(0xffffffffu, mc, o));
    }
    if (q == 0) {
        unsigned long long* rm = rmax + P * np;
        atomicMax(rm + I * 64 + k, (unsigned long long)__double_as_longlong(mr));
        if (I != J) atomicMax(rm + J * 64 + k, (unsigned long long)__double_as_longlong(mc));
    }
}

// Be[i] = e with max |row| 2^-e < 1 (0 for a zero row)
__global__ void row_exponent_kernel(const unsigned long long* __restrict__ rmax, long long count, int* __restrict__ Be) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double mx = __longlong_as_double((long long)rmax[i]);
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    Be[i] = e;
}

// slices of rows [0, nrows) of B (pointer at the block's first row): each packed tile (I, J) is read
// once and written as block (I, J) and, for I > J, transposed as block (J, I); Be holds the block's rows
template <int S>
__global__ void __launch_bounds__(256) split_b_tiles_kernel(const double* __restrict__ B, long long row, int np,
                                                            const int* __restrict__ Be, bf16* __restrict__ Bs,
                                                            long long sstride) {
    __shared__ double tile[64][65];
    const long long tp = blockIdx.x, P = blockIdx.y;
    int I, J;
    tile_of(tp, I, J);
    const double* src = B + P * row + tp * 4096;
    for (int i = threadIdx.x; i < 4096; i += 256) tile[i >> 6][i & 63] = src[i];
    __syncthreads();
    const int* e = Be + P * np;
    bf16* out = Bs + P * np * (long long)np;
    for (int i = threadIdx.x; i < 4096; i += 256) {   // block (I, J): mu = I*64 + r, nu = J*64 + c
        const int r = i >> 6, c = i & 63;
        const int mu = I * 64 + r;
        split_pow2<S>(tile[r][c], e[mu], out + (long long)mu * np + J * 64 + c, sstride);
    }
    if (I != J)
        for (int i = threadIdx.x; i < 4096; i += 256) {   // block (J, I): mu = J*64 + c, nu = I*64 + r
            const int r = i & 63, c = i >> 6;
            const int mu = J * 64 + c;
            split_pow2<S>(tile[r][c], e[mu], out + (long long)mu * np + I * 64 + r, sstride);
        }
}

// pmax[P] = max |B_P| as the bit pattern of a non-negative double, tile by tile
__global__ void __launch_bounds__(256) p_max_tiles_kernel(const double* __restrict__ B, long long row,
                                                          unsigned long long* __restrict__ pmax) {
    const long long tp = blockIdx.x, P = blockIdx.y;
    const double* src = B + P * row + tp * 4096;
    double m = 0.0;
    for (int i = threadIdx.x; i < 4096; i += 256) m = fmax(m, fabs(src[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(pmax + P, (unsigned long long)__double_as_longlong(m));
}

// slices of rows [0, nrows) of B into the packed layout Bs[s][P][t][128][128] (lower 128-tiles
// t = I (I + 1) / 2 + J, I >= J), one exponent Be[P] per row: the packed 64-tile (i, j) is block
// (i % 2, j % 2) of 128-tile (i / 2, j / 2); inside a diagonal 128-tile the off-diagonal 64-tile is also
// written transposed, so that diagonal tiles are whole. Blocks no 64-tile reaches (padding) stay as set
// at allocation (zero).
template <int S>
__global__ void __launch_bounds__(256) split_b_packed_kernel(const double* __restrict__ B, long long row,
                                                             const int* __restrict__ Be, long long ntile,
                                                             bf16* __restrict__ Bs, long long sstride) {
    __shared__ double tile[64][65];
    const long long tp = blockIdx.x, P = blockIdx.y;
    int I, J;
    tile_of(tp, I, J);
    const double* src = B + P * row + tp * 4096;
    for (int i = threadIdx.x; i < 4096; i += 256) tile[i >> 6][i & 63] = src[i];
    __syncthreads();
    const int e = Be[P];
    const int IB = I >> 1, JB = J >> 1;
    bf16* out = Bs + (P * ntile + (long long)IB * (IB + 1) / 2 + JB) * 16384;
    const int ro = (I & 1) * 64, co = (J & 1) * 64;
    for (int i = threadIdx.x; i < 4096; i += 256) {
        const int r = i >> 6, c = i & 63;
        split_pow2<S>(tile[r][c], e, out + (ro + r) * 128 + co + c, sstride);
    }
    if (IB == JB && I != J)
        for (int i = threadIdx.x; i < 4096; i += 256) {
            const int r = i & 63, c = i >> 6;
            split_pow2<S>(tile[r][c], e, out + (co + c) * 128 + ro + r, sstride);
        }
}

// C (n x nocc row-major) -> Cs[s][i][nu] (ldy x np), exponent per column i
template <int S>
__global__ void __launch_bounds__(256) split_c_kernel(const double* __restrict__ C, int n, int nocc, int np, int ldy,
                                                      bf16* __restrict__ Cs, long long sstride,
                                                      int* __restrict__ Ce) {
    const int i = blockIdx.x;
    double mx = 0.0;
    if (i < nocc)
        for (int nu = threadIdx.x; nu < n; nu += blockDim.x) mx = fmax(mx, fabs(C[(long long)nu * nocc + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);
    if (threadIdx.x == 0) Ce[i] = e;
    for (int nu = threadIdx.x; nu < np; nu += blockDim.x) {
        const double x = (i < nocc && nu < n) ? C[(long long)nu * nocc + i] : 0.0;
        split_pow2<S>(x, e, Cs + (long long)i * np + nu, sstride);
    }
}

// ------------------------------------------------------------------------------------------------
// Shared GEMM core: a CTA of WM x WN warps, warp tile 32 x 32; A rows and B rows (= output columns)
// both K-contiguous in global memory with leading dimensions lda, ldb. Per k-tile the CTA stages the
// S slices of A (BM x KT) and of B (BN x KT) and accumulates level accumulators acc[L-2].
// ------------------------------------------------------------------------------------------------
// warp tile 32 x (8 NJ): NJ = 4 for S <= 3, 2 for S >= 4 (keeps the S level accumulators in registers)
template <int S>
struct Frag {
    static constexpr int NJ = S <= 3 ? 4 : 2;
    float acc[S][2][NJ][4];   // [level][m16][n8][4]
    float hi[2][NJ][4], lo[2][NJ][4];
};

template <int S>
__device__ __forceinline__ void zero_acc(Frag<S>& f) {
#pragma unroll
    for (int L = 0; L < S; ++L)
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < Frag<S>::NJ; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) f.acc[L][a][b][c] = 0.f;
}

template <int S>
__device__ __forceinline__ void zero_hilo(Frag<S>& f) {
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < Frag<S>::NJ; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) f.hi[a][b][c] = f.lo[a][b][c] = 0.f;
}

// stage one k-tile of all slices: A rows [0, BM), B rows [0, BN), cp.async 16-byte pieces
template <int S>
__device__ __forceinline__ void stage_tile(bf16* sA, bf16* sB, const bf16* A, long long lda, long long astr,
                                           int a_rows, const bf16* Bm, long long ldb, long long bstr, int b_rows,
                                           int k0) {
    const int pieces_a = S * a_rows * (KT / 8);
    for (int p = threadIdx.x; p < pieces_a; p += blockDim.x) {
        const int s = p / (a_rows * (KT / 8));
        const int rem = p % (a_rows * (KT / 8));
        const int r = rem / (KT / 8), c = (rem % (KT / 8)) * 8;
        cp_async16(sA + (s * a_rows + r) * LDS + c, A + s * astr + r * lda + k0 + c);
    }
    const int pieces_b = S * b_rows * (KT / 8);
    for (int p = threadIdx.x; p < pieces_b; p += blockDim.x) {
        const int s = p / (b_rows * (KT / 8));
        const int rem = p % (b_rows * (KT / 8));
        const int r = rem / (KT / 8), c = (rem % (KT / 8)) * 8;
        cp_async16(sB + (s * b_rows + r) * LDS + c, Bm + s * bstr + r * ldb + k0 + c);
    }
}

// MMAs of one staged k-tile: warp (wm, wn) covers A rows wm*32.., B rows wn*WNT..
template <int S>
__device__ __forceinline__ void mma_tile(Frag<S>& f, const bf16* sA, int a_rows, const bf16* sB, int b_rows, int wm,
                                         int wn, int lane) {
#pragma unroll
    for (int kk = 0; kk < KT; kk += 16) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            unsigned afr[2][4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const bf16* p = sA + (s * a_rows + wm * 32 + mi * 16 + (lane & 15)) * LDS + kk + (lane >> 4) * 8;
                ldmatrix_x4(afr[mi], p);
            }
#pragma unroll
            for (int t = 0; t < S - s; ++t) {   // s + t <= S - 1 (0-based) <=> level s + t + 2 <= S + 1
                constexpr int NJ = Frag<S>::NJ;
                unsigned bfr[NJ][2];
#pragma unroll
                for (int j = 0; j < NJ; j += 2) {
                    const int q = lane >> 3, r = lane & 7;
                    const bf16* p = sB + (t * b_rows + wn * NJ * 8 + (j + (q >> 1)) * 8 + r) * LDS + kk + (q & 1) * 8;
                    unsigned v[4];
                    ldmatrix_x4(v, p);
                    bfr[j][0] = v[0];
                    bfr[j][1] = v[1];
                    bfr[j + 1][0] = v[2];
                    bfr[j + 1][1] = v[3];
                }
#pragma unroll
                for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                    for (int j = 0; j < NJ; ++j) mma_bf16(f.acc[s + t][mi][j], afr[mi], bfr[j]);
            }
        }
    }
}

// drain: hi/lo += acc[L] * 2^{ea(row) + eb(col) - 7 (L + 2)}, then acc = 0
template <int S>
__device__ __forceinline__ void drain(Frag<S>& f, const int* ea, const int* eb, int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int er = ea[mi * 16 + g + 8 * h];
#pragma unroll
            for (int j = 0; j < Frag<S>::NJ; ++j)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int ec = eb[j * 8 + 2 * t + c];
                    // levels are combined with exact power-of-two factors; smaller levels are added last
#pragma unroll
                    for (int L = S - 1; L >= 0; --L) {
                        const float x = f.acc[L][mi][j][2 * h + c] * pow2f(er + ec - 7 * (L + 2));
                        two_sum_acc(f.hi[mi][j][2 * h + c], f.lo[mi][j][2 * h + c], x);
                        f.acc[L][mi][j][2 * h + c] = 0.f;
                    }
                }
        }
}

// ------------------------------------------------------------------------------------------------
// Y = B_P C (split): CTA = P, 64 rows mu, 32*WN columns i; output (hi, lo) pairs Y[P][mu][i]
// ------------------------------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(320) y_split_kernel(const bf16* __restrict__ Bs, long long bstr,
                                                      const int* __restrict__ Be, const bf16* __restrict__ Cs,
                                                      long long cstr, const int* __restrict__ Ce, int np, int ldy,
                                                      float2* __restrict__ Y) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int WNT = 8 * Frag<S>::NJ;
    const int WN = blockDim.x / 64;
    const int BN = WNT * WN;
    bf16* sA = reinterpret_cast<bf16*>(smem_raw);                 // [2][S][64][LDS]
    bf16* sB = sA + 2 * S * 64 * LDS;                               // [2][S][BN][LDS]
    int* sEa = reinterpret_cast<int*>(sB + 2 * S * BN * LDS);       // [64]
    int* sEb = sEa + 64;                                            // [BN]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp & 1, wn = warp >> 1;
    const int m0 = blockIdx.x * 64;
    const int n0 = blockIdx.z * BN;
    const long long P = blockIdx.y;
    const bf16* A = Bs + (P * np + m0) * (long long)np;
    const bf16* Bm = Cs + (long long)n0 * np;
    for (int r = threadIdx.x; r < 64; r += blockDim.x) sEa[r] = Be[P * np + m0 + r];
    for (int c = threadIdx.x; c < BN; c += blockDim.x) sEb[c] = (n0 + c < ldy) ? Ce[n0 + c] : 0;
    const int b_rows = min(BN, ldy - n0);
    Frag<S> f;
    zero_acc(f);
    zero_hilo(f);
    const int nk = np / KT;
    stage_tile<S>(sA, sB, A, np, bstr, 64, Bm, np, cstr, b_rows, 0);
    cp_async_commit();
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk)
            stage_tile<S>(sA + (cur ^ 1) * S * 64 * LDS, sB + (cur ^ 1) * S * BN * LDS, A, np, bstr, 64, Bm, np, cstr,
                          b_rows, (kt + 1) * KT);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        if (wn * WNT < b_rows) mma_tile<S>(f, sA + cur * S * 64 * LDS, 64, sB + cur * S * BN * LDS, BN, wm, wn, lane);
        __syncthreads();
        if ((kt + 1) % (exact_chunk<S>() / KT) == 0 || kt + 1 == nk) drain<S>(f, sEa + wm * 32, sEb + wn * WNT, lane);
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int mu = m0 + wm * 32 + mi * 16 + g + 8 * h;
#pragma unroll
            for (int j = 0; j < Frag<S>::NJ; ++j)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int i = n0 + wn * WNT + j * 8 + 2 * t + c;
                    if (i < ldy) Y[(P * np + mu) * (long long)ldy + i] = make_float2(f.hi[mi][j][2 * h + c], f.lo[mi][j][2 * h + c]);
                }
        }
}

// Y (hi, lo) -> Ys[s][P][mu][i] with one exponent per (mu, block of PB auxiliary rows); warp per (mu, block)
template <int S>
__global__ void __launch_bounds__(256) split_y_kernel(const float2* __restrict__ Y, int naux, int np, int ldy, int PB,
                                                      bf16* __restrict__ Ys, long long sstride, int* __restrict__ Ye) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nblk = (naux + PB - 1) / PB;
    if (warp >= nblk * np) return;
    const int mu = warp % np, b = warp / np;
    const int p0 = b * PB, p1 = min(naux, p0 + PB);
    float mx = 0.f;
    for (int P = p0; P < p1; ++P)
        for (int i = lane; i < ldy; i += 32) mx = fmaxf(mx, fabsf(Y[((long long)P * np + mu) * ldy + i].x));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);   // |hi + lo| 2^-e <= 1 + 2^-24, so |m_1| <= 128 still holds
    if (lane == 0) Ye[(long long)b * np + mu] = e;
    const float sc = pow2f(-e);
    for (int P = p0; P < p1; ++P)
        for (int i = lane; i < ldy; i += 32) {
            const long long idx = ((long long)P * np + mu) * ldy + i;
            const float2 y = Y[idx];
            float r = y.x * sc;
            float rl = y.y * sc;
            bf16* out = Ys + idx;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const float tt = r * 128.f;
                const float m = rintf(tt);
                r = (tt - m) + rl * 128.f;
                rl = 0.f;
                out[s * sstride] = __float2bfloat16_rn(m);
            }
        }
}

// Y (hi, lo) -> Ys over the contiguous contraction index k = P ldy + i (KL = naux ldy values per row mu), one
// exponent per (mu, chunk of CH consecutive k): the operand layout of the tensor-core exchange contraction.
// Tile-major: Ys[s][k / 64][mu][k % 64], so that one TMA box (128 rows x 64 k) is 16 KB of contiguous memory;
// no padding between auxiliary rows; the tail of the last 64-block (k >= KL) is zero. Warp per (mu, chunk).
template <int S>
__global__ void __launch_bounds__(256) split_y_rows_kernel(const float2* __restrict__ Y, int np, int ldy, long long KL,
                                                           int CH, bf16* __restrict__ Ys, int* __restrict__ Ye) {
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long nchk = (KL + CH - 1) / CH;
    if (warp >= nchk * np) return;
    const int mu = (int)(warp % np);
    const long long b = warp / np;
    const long long k0 = b * CH, k1 = min(KL, k0 + CH);
    const long long nkb = (KL + 63) / 64;
    const long long sstride = nkb * np * 64;
    // the chunk's k run over auxiliary rows P0, P0 + 1, ...: one division per warp, then per-row segments
    const long long P0 = k0 / ldy;
    const int i0 = (int)(k0 - P0 * ldy);
    float mx = 0.f;
    {
        long long k = k0, P = P0;
        int i = i0;
        while (k < k1) {
            const int seg = (int)min((long long)(ldy - i), k1 - k);
            const float2* y = Y + (P * np + mu) * ldy + i;
            for (int j = lane; j < seg; j += 32) mx = fmaxf(mx, fabsf(y[j].x));
            k += seg;
            ++P;
            i = 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);   // |hi + lo| 2^-e <= 1 + 2^-24, so |m_1| <= 128 still holds
    if (lane == 0) Ye[b * np + mu] = e;
    const float sc = pow2f(-e);
    long long k = k0, P = P0;
    int i = i0;
    while (k < k1) {
        const int seg = (int)min((long long)(ldy - i), k1 - k);
        const float2* y = Y + (P * np + mu) * ldy + i;
        for (int j = lane; j < seg; j += 32) {
            const float2 v = y[j];
            const long long kk = k + j;
            bf16* out = Ys + ((kk >> 6) * np + mu) * 64 + (kk & 63);
            float r = v.x * sc;
            float rl = v.y * sc;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const float tt = r * 128.f;
                const float m = rintf(tt);
                r = (tt - m) + rl * 128.f;
                rl = 0.f;
                out[s * sstride] = __float2bfloat16_rn(m);
            }
        }
        k += seg;
        ++P;
        i = 0;
    }
    if (k1 == KL)   // the warps of the last chunk zero the tail of the last 64-block
        for (long long kk = KL + lane; kk < nkb * 64; kk += 32) {
            bf16* out = Ys + ((kk >> 6) * np + mu) * 64 + (kk & 63);
#pragma unroll
            for (int s = 0; s < S; ++s) out[s * sstride] = __float2bfloat16_rn(0.f);
        }
}

// ------------------------------------------------------------------------------------------------
// K partial sums over a range of auxiliary blocks for lower tile pair (I >= J) of 64 x 64
// ------------------------------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(256) k_split_kernel(const bf16* __restrict__ Ys, long long sstride,
                                                      const int* __restrict__ Ye, int naux, int np, int ldy, int PB,
                                                      int nsplit, const int2* __restrict__ tiles,
                                                      float2* __restrict__ Kpart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16* sA = reinterpret_cast<bf16*>(smem_raw);     // [2][S][64][LDS]
    bf16* sB = sA + 2 * S * 64 * LDS;                 // [2][S][64][LDS]
    __shared__ int sEa[64], sEb[64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp & 1, wn = warp >> 1;
    const int2 IJ = tiles[blockIdx.x];
    const int nblk = (naux + PB - 1) / PB;
    const int b0 = (int)((long long)nblk * blockIdx.y / nsplit), b1 = (int)((long long)nblk * (blockIdx.y + 1) / nsplit);
    constexpr int WNT = 8 * Frag<S>::NJ;
    Frag<S> f;
    zero_acc(f);
    zero_hilo(f);
    const int kt_per_P = ldy / KT;
    for (int blk = b0; blk < b1; ++blk) {
        const int p0 = blk * PB, p1 = min(naux, p0 + PB);
        __syncthreads();
        for (int r = threadIdx.x; r < 64; r += blockDim.x) {
            sEa[r] = Ye[(long long)blk * np + IJ.x * 64 + r];
            sEb[r] = Ye[(long long)blk * np + IJ.y * 64 + r];
        }
        const int nk = (p1 - p0) * kt_per_P;
        auto src = [&](int kt, int rowtile) {
            const int P = p0 + kt / kt_per_P;
            return Ys + ((long long)P * np + rowtile * 64) * ldy + (kt % kt_per_P) * KT;
        };
        stage_tile<S>(sA, sB, src(0, IJ.x), ldy, sstride, 64, src(0, IJ.y), ldy, sstride, 64, 0);
        cp_async_commit();
        for (int kt = 0; kt < nk; ++kt) {
            const int cur = kt & 1;
            if (kt + 1 < nk)
                stage_tile<S>(sA + (cur ^ 1) * S * 64 * LDS, sB + (cur ^ 1) * S * 64 * LDS, src(kt + 1, IJ.x), ldy,
                              sstride, 64, src(kt + 1, IJ.y), ldy, sstride, 64, 0);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            mma_tile<S>(f, sA + cur * S * 64 * LDS, 64, sB + cur * S * 64 * LDS, 64, wm, wn, lane);
            __syncthreads();
        }
        drain<S>(f, sEa + wm * 32, sEb + wn * WNT, lane);
    }
    float2* Kp = Kpart + (long long)blockIdx.y * np * np;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int mu = IJ.x * 64 + wm * 32 + mi * 16 + g + 8 * h;
#pragma unroll
            for (int j = 0; j < Frag<S>::NJ; ++j)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int nu = IJ.y * 64 + wn * WNT + j * 8 + 2 * t + c;
                    Kp[(long long)mu * np + nu] = make_float2(f.hi[mi][j][2 * h + c], f.lo[mi][j][2 * h + c]);
                }
        }
}

__global__ void k_split_reduce_kernel(const float2* __restrict__ Kpart, int nsplit, int np, int n, double* __restrict__ K) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    int a = (int)(idx / n), b = (int)(idx % n);
    if (a / 64 < b / 64) { const int t = a; a = b; b = t; }
    double s = 0.0;
    for (int q = 0; q < nsplit; ++q) {
        const float2 v = Kpart[(long long)q * np * np + (long long)a * np + b];
        s += (double)v.x + (double)v.y;
    }
    K[idx] = s;
}

inline unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// tcgen05 kernels for the split products (3 and 5 slices); DFHF_SPLIT_TC=0 selects the mma.sync kernels
bool use_tensor_cores() {
    const char* v = std::getenv("DFHF_SPLIT_TC");
    return !(v && v[0] == '0');
}

// B slice layout for the tensor-core Y: full rows (one exponent per (P, mu): the smaller splitting error)
// when every row's slices fit in HBM, else packed lower 128-tiles (half the memory: 40 waters keep every
// slice resident); DFHF_TC_PACKED=1 / 0 forces packed / full rows (tests compare the two). Returns 1, 0, or
// -1 for the automatic choice.
int packed_preference() {
    const char* v = std::getenv("DFHF_TC_PACKED");
    if (v && v[0] == '1') return 1;
    if (v && v[0] == '0') return 0;
    return -1;
}

}  // namespace

void y_split_tc(cudaStream_t s, int S, int N, const bf16* Bs, const int* Be, const bf16* Cs, const int* Ce, int naux,
                int np, int ldy, float2* Y, int* err);
void y_split_tc_packed(cudaStream_t s, int S, int N, const bf16* Bs, const int* Be, const bf16* Cs, const int* Ce,
                       int naux, int zrows, int np, int nB, int ldy, float2* Y, int* err);
void k_split_tc(cudaStream_t s, int S, int N, const bf16* Ys, const int* Ye, int naux, int np, int ldy, int nsplit,
                const int2* tiles128, int ntiles, float2* Kpart, int npt, int* err);
void k_tc_reduce(cudaStream_t s, const float2* Kpart, int nsplit, int npt, int n, double* K);

struct SplitState {
    // tensor-core (tcgen05) path
    int* err = nullptr;          // device error word of the tcgen05 kernels
    int2* tiles128 = nullptr;    // lower 128-tile pairs
    float2* Kpart_tc = nullptr;  // [nsplit_tc][npt][npt]
    int npt = 0, ntiles128 = 0, nsplit_tc = 0, kcap = 0;   // kcap: splits Kpart_tc has room for
    int ksplit_heur = 1;         // K split of the occupancy heuristic (about 4 CTAs per SM)
    int yN = 80;                 // tile width of the tensor-core Y kernel
    int kN = 64;                 // half-tile width of the tensor-core K kernel
    int S = 0;
    int np = 0;
    bf16* Bs = nullptr;
    int* Be = nullptr;
    bf16* Cs = nullptr;
    int* Ce = nullptr;
    float2* Y = nullptr;
    bf16* Ys = nullptr;
    int* Ye = nullptr;
    float2* Kpart = nullptr;
    int ldy = 0;
    int ldy_cap = 0;             // occupied width the Cs, Ce, Y and Ys buffers were sized for
    long long ye_cap = 0;        // entries of Ye
    int kpart_cap = 0;           // splits Kpart has room for (mma.sync contraction)
    int nsplit = 0;
    int PB = 0;
    bool blocked = false;        // B slices cut per block of pblk auxiliary rows at every build
    int pblk = 0;
    // B slice layout: tensor-core path packed lower 128-tiles with one exponent per auxiliary row
    // (Bs [S][rows][nB (nB + 1) / 2][128][128], Be [naux]); mma.sync path full rows with one exponent per
    // (P, mu) (Bs [S][rows][np][np], Be [naux][np])
    bool packed = false;
    int nB = 0;
    long long ntile = 0;
    // tile choice per slice count, fixed at this state's first build with that count (0: not yet):
    // Y tile width, K tile width, K split; buffers sized for it are never reallocated under queued work
    int ch_y[SMAX + 1] = {0}, ch_k[SMAX + 1] = {0}, ch_split[SMAX + 1] = {0};
};

void free_split(df_handle* h) {
    SplitState* st = h->split;
    if (!st) return;
    cudaStreamSynchronize(h->stream);   // queued builds finish before their buffers go
    cudaFree(st->Bs);
    cudaFree(st->Be);
    cudaFree(st->Cs);
    cudaFree(st->Ce);
    cudaFree(st->Y);
    cudaFree(st->Ys);
    cudaFree(st->Ye);
    cudaFree(st->Kpart);
    cudaFree(st->err);
    cudaFree(st->tiles128);
    cudaFree(st->Kpart_tc);
    delete st;
    h->split = nullptr;
}

namespace {

// exponent of every row (P, mu) of B, from the packed tiles (B does not change for the handle)
void row_exponents(df_handle* h, SplitState* st) {
    if (h->naux > 65535) throw Error{DF_E_ARG, "split exchange supports at most 65535 auxiliary functions"};
    const long long count = (long long)h->naux * st->np;
    DF_CUDA(cudaMalloc((void**)&st->Be, sizeof(int) * count));
    DevBuf<unsigned long long> rmax;
    rmax.alloc(count);
    rmax.zero(h->stream);
    row_max_tiles_kernel<<<dim3((unsigned)h->pk.ntp, h->naux), 256, 0, h->stream>>>(h->B.p, h->pk.row, st->np, rmax.p);
    DF_CHECK_LAUNCH();
    row_exponent_kernel<<<nblocks(count, 256), 256, 0, h->stream>>>(rmax.p, count, st->Be);
    DF_CHECK_LAUNCH();
    DF_CUDA(cudaStreamSynchronize(h->stream));   // rmax is released on return
}

// one exponent per auxiliary row P (packed layout): max over B_P
void p_exponents(df_handle* h, SplitState* st) {
    if (h->naux > 65535) throw Error{DF_E_ARG, "split exchange supports at most 65535 auxiliary functions"};
    DF_CUDA(cudaMalloc((void**)&st->Be, sizeof(int) * h->naux));
    DevBuf<unsigned long long> pmax;
    pmax.alloc(h->naux);
    pmax.zero(h->stream);
    p_max_tiles_kernel<<<dim3((unsigned)h->pk.ntp, h->naux), 256, 0, h->stream>>>(h->B.p, h->pk.row, pmax.p);
    DF_CHECK_LAUNCH();
    row_exponent_kernel<<<nblocks(h->naux, 256), 256, 0, h->stream>>>(pmax.p, h->naux, st->Be);
    DF_CHECK_LAUNCH();
    DF_CUDA(cudaStreamSynchronize(h->stream));   // pmax is released on return
}

// elements of one auxiliary row's slices in the state's layout
long long row_elems(const SplitState* st) { return st->packed ? st->ntile * 16384 : (long long)st->np * st->np; }

// the slice buffer for `rows` auxiliary rows (zeroed: the packed layout's padding is never written)
void alloc_b_slices(df_handle* h, SplitState* st, long long rows) {
    const long long elems = (long long)SMAX * rows * row_elems(st);
    DF_CUDA(cudaMalloc((void**)&st->Bs, sizeof(bf16) * elems));
    if (st->packed) DF_CUDA(cudaMemsetAsync(st->Bs, 0, sizeof(bf16) * elems, h->stream));
}

void b_exponents(df_handle* h, SplitState* st) {
    if (st->packed) p_exponents(h, st);
    else row_exponents(h, st);
}

// slices of auxiliary rows [p0, p0 + nb) into Bs (block-local rows; bstr = elements per slice)
template <int S>
void slice_b_rows(df_handle* h, SplitState* st, int p0, int nb, long long bstr) {
    if (st->packed)
        split_b_packed_kernel<S><<<dim3((unsigned)h->pk.ntp, nb), 256, 0, h->stream>>>(
            h->B.p + (long long)p0 * h->pk.row, h->pk.row, st->Be + p0, st->ntile, st->Bs, bstr);
    else
        split_b_tiles_kernel<S><<<dim3((unsigned)h->pk.ntp, nb), 256, 0, h->stream>>>(
            h->B.p + (long long)p0 * h->pk.row, h->pk.row, st->np, st->Be + (long long)p0 * st->np, st->Bs, bstr);
    DF_CHECK_LAUNCH();
}

template <int S>
void prepare_b(df_handle* h, SplitState* st) {
    alloc_b_slices(h, st, h->naux);
    b_exponents(h, st);
    slice_b_rows<S>(h, st, 0, h->naux, (long long)h->naux * row_elems(st));
}

// ---- autotuner ----------------------------------------------------------------------------------
// The tile width of the tensor-core Y kernel (32, 64 or 80 columns dividing ldy) and of the K kernel (32
// or 64) are picked by timing the candidates on the call's own operands the first time a size bucket
// (np, ldy, naux / 512, S) is met; the choice is kept for the process. Y is timed on the first auxiliary
// block (all rows when every slice is resident), K on the finished Y slices. Every width computes the
// same values bit for bit; the K split over auxiliary blocks comes from the occupancy heuristic.
struct TcChoice {
    int yN = 0, kN = 64, ksplit = 0;
};
std::mutex g_tune_mu;
std::map<std::array<int, 4>, TcChoice> g_tune;
double g_tune_ms = 0.0;

template <typename F>
double time_once(cudaStream_t s, F&& launch) {
    cudaEvent_t a, b;
    DF_CUDA(cudaEventCreate(&a));
    DF_CUDA(cudaEventCreate(&b));
    launch();   // warm-up: first-launch attribute and module set-up
    DF_CUDA(cudaEventRecord(a, s));
    launch();
    DF_CUDA(cudaEventRecord(b, s));
    DF_CUDA(cudaEventSynchronize(b));
    const double ms = elapsed_ms(a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

// tensor-core Y of auxiliary rows [p0, p0 + nb) held in the slice buffer (block-local rows)
void y_tc(df_handle* h, SplitState* st, int S, int N, int p0, int nb, float2* Yb) {
    if (st->packed)   // slices at the buffer's full row stride (the padding of every block stays zero)
        y_split_tc_packed(h->stream, S, N, st->Bs, st->Be + p0, st->Cs, st->Ce, nb, st->blocked ? st->pblk : h->naux,
                          st->np, st->nB, st->ldy, Yb, st->err);
    else
        y_split_tc(h->stream, S, N, st->Bs, st->Be + (long long)p0 * st->np, st->Cs, st->Ce, nb, st->np, st->ldy, Yb,
                   st->err);
}

template <int S>
int tune_y(df_handle* h, SplitState* st, int nb, float2* Yb) {
    double best_ms = 1e30;
    int best = 0;
    for (int N : {80, 64, 32}) {
        if (st->ldy % N) continue;
        const double ms = time_once(h->stream, [&] { y_tc(h, st, S, N, 0, nb, Yb); });
        if (ms < best_ms) {
            best_ms = ms;
            best = N;
        }
    }
    return best;
}

template <int S>
void tune_k(df_handle* h, SplitState* st, TcChoice& best) {
    cudaStream_t s = h->stream;
    const int np = st->np, ldy = st->ldy, naux = h->naux;
    const long long nblk = ((long long)naux * ldy + exact_chunk<S>() - 1) / exact_chunk<S>();
    const int h0 = std::max(1, (int)std::min<long long>(st->ksplit_heur, nblk));   // occupancy heuristic
    if (h0 > st->kcap) {
        DF_CUDA(cudaStreamSynchronize(s));
        cudaFree(st->Kpart_tc);
        st->Kpart_tc = nullptr;
        DF_CUDA(cudaMalloc((void**)&st->Kpart_tc, sizeof(float2) * h0 * (long long)st->npt * st->npt));
        st->kcap = h0;
    }
    // the half-tile width at the heuristic's split
    double best_ms = 1e30;
    for (int N : {64, 32}) {
        const double ms = time_once(s, [&] {
            k_split_tc(s, S, N, st->Ys, st->Ye, naux, np, ldy, h0, st->tiles128, st->ntiles128, st->Kpart_tc,
                       st->npt, st->err);
        });
        if (ms < best_ms) {
            best_ms = ms;
            best.kN = N;
        }
    }
    // the split changes how the float-float partial sums are grouped (hence the last bits of K), so it
    // is not chosen by timing: the occupancy heuristic keeps results identical from run to run
    best.ksplit = h0;
}

// Y over auxiliary blocks: one block of all rows when every slice is resident; otherwise the slices of
// each block of st->pblk rows are cut from the packed FP64 B just before the Y kernel consumes them.
template <int S>
void run_split(df_handle* h, SplitState* st, const double* dC, int nocc, double* dK, PhaseTimer& ev) {
    cudaStream_t s = h->stream;
    const int np = st->np, ldy = st->ldy, naux = h->naux;
    const long long cstr = (long long)ldy * np;
    split_c_kernel<S><<<ldy, 256, 0, s>>>(dC, h->n, nocc, np, ldy, st->Cs, cstr, st->Ce);
    DF_CHECK_LAUNCH();
    // mma.sync Y: CTA tiles of 64 rows x 32*WN columns
    constexpr int WNT = 8 * Frag<S>::NJ;
    const int WN = std::min(5, ldy / WNT);
    const int BN = WNT * WN;
    const size_t smem = (size_t)2 * S * (64 + BN) * LDS * sizeof(bf16) + (64 + BN) * sizeof(int);
    DF_CUDA(cudaFuncSetAttribute(y_split_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const bool tc = use_tensor_cores() && (S == 3 || S == 5);
    if (st->packed && !tc) throw Error{DF_E_ARG, "internal: B slice layout does not match the exchange kernels"};
    const std::array<int, 4> key{np, ldy, (naux + 511) / 512, S};
    TcChoice ch;
    bool have = !tc;
    // DFHF_TC_TILES="yN,kN,ksplit" fixes the choice (tests compare tilings; the results do not depend on it)
    if (const char* f = tc ? std::getenv("DFHF_TC_TILES") : nullptr) {
        TcChoice fc;
        if (std::sscanf(f, "%d,%d,%d", &fc.yN, &fc.kN, &fc.ksplit) == 3 && fc.ksplit >= 1 &&
            (fc.yN == 32 || fc.yN == 64 || fc.yN == 80) && ldy % fc.yN == 0 && (fc.kN == 32 || fc.kN == 64)) {
            ch = fc;
            have = true;
        }
    }
    if (tc && !have && st->ch_y[S]) {   // this state's own choice: stable across its builds
        ch.yN = st->ch_y[S];
        ch.kN = st->ch_k[S];
        ch.ksplit = st->ch_split[S];
        have = true;
    } else if (tc && !have) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            ch = it->second;
            have = true;
        }
    }
    double tune_ms = 0.0;
    ev.mark(1, s);
    const int pblk = st->blocked ? st->pblk : naux;
    for (int p0 = 0; p0 < naux; p0 += pblk) {
        const int nb = std::min(pblk, naux - p0);
        // slice stride: the packed layout keeps the buffer's full row count, so that the zero padding of
        // the last 128-tiles sits at the same place for every block
        const long long bstr = (long long)(st->blocked ? (st->packed ? st->pblk : nb) : naux) * row_elems(st);
        if (st->blocked) slice_b_rows<S>(h, st, p0, nb, bstr);
        const int* Beb = st->Be + (long long)p0 * np;   // row exponents of the block (mma.sync layout)
        float2* Yb = st->Y + (long long)p0 * np * ldy;
        if (tc) {
            if (!have && p0 == 0) {
                const auto t0 = std::chrono::steady_clock::now();
                ch.yN = tune_y<S>(h, st, nb, Yb);
                tune_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            }
            y_tc(h, st, S, ch.yN, p0, nb, Yb);
        } else {
            y_split_kernel<S><<<dim3(np / 64, nb, (ldy + BN - 1) / BN), 64 * WN, smem, s>>>(st->Bs, bstr, Beb, st->Cs,
                                                                                           cstr, st->Ce, np, ldy, Yb);
            DF_CHECK_LAUNCH();
        }
    }
    ev.mark(2, s);
    {
        const int nyb = (naux + pblk - 1) / pblk;   // split C, per block (slicing,) Y, re-split Y, K, reduce
        h->exchange_launches = 4 + nyb * (st->blocked ? 2 : 1);
    }
    const long long ystr = (long long)naux * np * ldy;
    // the tensor-core contraction takes Ys[s][k / 64][mu][k % 64] (k = P ldy + i, chunks of the exact length
    // for S); the
    // mma.sync contraction Ys[s][P][mu][i] with chunks of PB auxiliary rows
    const long long nblk = tc ? ((long long)naux * ldy + exact_chunk<S>() - 1) / exact_chunk<S>()
                              : (naux + st->PB - 1) / st->PB;
    if (tc)
        split_y_rows_kernel<S><<<nblocks(nblk * np * 32, 256), 256, 0, s>>>(st->Y, np, ldy, (long long)naux * ldy,
                                                                           exact_chunk<S>(), st->Ys, st->Ye);
    else
        split_y_kernel<S><<<nblocks(nblk * np * 32, 256), 256, 0, s>>>(st->Y, naux, np, ldy, st->PB, st->Ys, ystr,
                                                                      st->Ye);
    DF_CHECK_LAUNCH();
    if (tc) {
        if (!have) {
            const auto t0 = std::chrono::steady_clock::now();
            tune_k<S>(h, st, ch);
            tune_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tune.emplace(key, ch);   // the first tuned choice of a bucket stays
            g_tune_ms += tune_ms;
        }
        // a choice made for another handle of the bucket: at most one split per exponent block, and room
        // for it in the partial-sum buffer
        // the override's split, else this state's own heuristic (a cached choice carries only widths)
        const int ksplit = (int)std::min<long long>(std::getenv("DFHF_TC_TILES") && ch.ksplit > 0 ? ch.ksplit
                                                                                                 : st->ksplit_heur,
                                                    nblk);
        st->ch_y[S] = ch.yN;
        st->ch_k[S] = ch.kN;
        st->ch_split[S] = ksplit;
        if (ksplit > st->kcap) {
            DF_CUDA(cudaStreamSynchronize(s));   // nothing queued may still read the old buffer
            cudaFree(st->Kpart_tc);
            st->Kpart_tc = nullptr;
            DF_CUDA(cudaMalloc((void**)&st->Kpart_tc, sizeof(float2) * ksplit * (long long)st->npt * st->npt));
            st->kcap = ksplit;
        }
        st->yN = ch.yN;
        st->kN = ch.kN;
        st->nsplit_tc = ksplit;
        h->timings_ms[12] = ch.yN;
        h->timings_ms[13] = ksplit;
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            h->timings_ms[14] = g_tune_ms;
        }
        h->timings_ms[15] = ch.kN;
        ev.mark(3, s);
        k_split_tc(s, S, ch.kN, st->Ys, st->Ye, naux, np, ldy, ksplit, st->tiles128, st->ntiles128, st->Kpart_tc,
                   st->npt, st->err);
        ev.mark(4, s);
        k_tc_reduce(s, st->Kpart_tc, ksplit, st->npt, h->n, dK);
    } else {
        const int nt = np / 64;
        const int ntiles = nt * (nt + 1) / 2;
        const size_t ksmem = (size_t)2 * 2 * S * 64 * LDS * sizeof(bf16);
        DF_CUDA(cudaFuncSetAttribute(k_split_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ksmem));
        ev.mark(3, s);
        k_split_kernel<S><<<dim3(ntiles, st->nsplit), 2 * (64 / WNT) * 32, ksmem, s>>>(
            st->Ys, ystr, st->Ye, naux, np, ldy, st->PB, st->nsplit, h->ktiles.p, st->Kpart);
        DF_CHECK_LAUNCH();
        ev.mark(4, s);
        const long long nn = (long long)h->n * h->n;
        k_split_reduce_kernel<<<nblocks(nn, 256), 256, 0, s>>>(st->Kpart, st->nsplit, np, h->n, dK);
        DF_CHECK_LAUNCH();
    }
}
}  // namespace

// K from the split path for the occupied coefficients dC (n x nocc, device).
// B is split once with SMAX slices when HBM allows, so that builds with fewer slices (early SCF
// iterations) and with SMAX slices (late iterations) share one split: the first S slices of an
// SMAX-slice split are an S-slice split of the same values (same exponents; within 0.51 2^{-7S} of
// each scaled value). Otherwise the slices are cut per block of auxiliary rows at every build.
void exchange_split(df_handle* h, const double* dC, int nocc, int slices, double* dK) {
    if (slices < 2 || slices > SMAX) throw Error{DF_E_ARG, "slices must be 2..5"};
    if (h->pk.np % 64) throw Error{DF_E_ARG, "internal: padded size not a multiple of 64"};
    SplitState* st = h->split;
    // the tensor-core kernels read the packed slice layout, the mma.sync kernels the full one: a build of the
    // other kind re-cuts the slices (tests switch kernels on one handle; an SCF stays with one kind)
    const bool tc_ok = use_tensor_cores() && (slices == 3 || slices == 5);
    const int pref = packed_preference();
    if (st && (st->S < slices || (st->packed && !tc_ok) || (pref >= 0 && st->packed != (tc_ok && pref == 1)))) {
        free_split(h);
        st = nullptr;
    }
    // phase marks: 0 start, 1-2 Y, 3-4 K contraction, 5 end
    PhaseTimer ev(h->sync_timing, 6);
    ev.mark(0, h->stream);
    const int ldy = ((nocc + 31) / 32) * 32;
    // set-up: a failure part-way leaves no half-built state behind (the next call starts afresh)
    try {
    if (!st) {
        st = new SplitState();
        h->split = st;
        st->np = h->pk.np;
        st->nB = (st->np + 127) / 128;
        st->ntile = (long long)st->nB * (st->nB + 1) / 2;
        const long long np = st->np;
        // FP64 builds on this handle borrow the split Y from now on: an FP64 Y already allocated goes
        if (h->Y.p) {
            DF_CUDA(cudaStreamSynchronize(h->stream));
            h->Y.release();
        }
        size_t free_b = 0, total_b = 0;
        DF_CUDA(cudaMemGetInfo(&free_b, &total_b));
        // SMAX slices of every auxiliary row when they fit beside Y and its slices; otherwise SMAX slices
        // of blocks of rows, cut from B at each build
        const double ybytes = (8.0 + 2.0 * SMAX) * h->naux * np * ldy;      // Y and its slices
        // kept free: working space (FP64 builds on the same handle use the split Y buffer)
        const double slack = 16.0 * np * np + (4ull << 30);
        if (!tc_ok) st->packed = false;
        else if (pref >= 0) st->packed = pref == 1;
        else st->packed = (double)free_b <= 2.0 * SMAX * np * np * h->naux + ybytes + slack;
        const double row_slices = 2.0 * SMAX * row_elems(st);                // one row, every slice
        st->S = SMAX;
        // DFHF_SPLIT_BLOCK_ROWS=r forces blocks of r rows (tests compare the two modes)
        const char* fb = std::getenv("DFHF_SPLIT_BLOCK_ROWS");
        const int forced = fb ? std::atoi(fb) : 0;
        if (forced > 0) {
            st->blocked = true;
            st->pblk = std::min(forced, h->naux);
            alloc_b_slices(h, st, st->pblk);
            b_exponents(h, st);
        } else if ((double)free_b > row_slices * h->naux + ybytes + slack) {
            prepare_b<SMAX>(h, st);
        } else {
            const double avail = (double)free_b - ybytes - slack;
            if (avail < row_slices) throw Error{DF_E_NOMEM, "split exchange: no room for one row of B slices"};
            st->blocked = true;
            st->pblk = (int)std::min<double>(h->naux, std::floor(avail / row_slices));
            alloc_b_slices(h, st, st->pblk);
            b_exponents(h, st);
        }
    }
    if (ldy != st->ldy) {
        DF_CUDA(cudaStreamSynchronize(h->stream));   // earlier builds may still read these buffers
        if (ldy > CHUNK_TILES * KT) throw Error{DF_E_ARG, "split exchange supports nocc <= 512"};
        st->ldy = ldy;
        // the tile choices were made for the previous occupied width (a width need not divide the new one)
        for (int q = 0; q <= SMAX; ++q) st->ch_y[q] = st->ch_k[q] = st->ch_split[q] = 0;
        st->PB = std::max(1, (CHUNK_TILES * KT) / ldy);
        const int nt = st->np / 64;
        const int ntiles = nt * (nt + 1) / 2;
        st->nsplit = std::max(1, std::min((8 * 152 + ntiles - 1) / ntiles, (h->naux + st->PB - 1) / st->PB));
        const long long np = st->np;
        // buffers keep the largest width met (an SCF from the SAD factor builds its first exchange wider):
        // a narrower build reuses them without reallocating
        if (ldy > st->ldy_cap) {
            cudaFree(st->Cs);
            cudaFree(st->Ce);
            cudaFree(st->Y);
            cudaFree(st->Ys);
            st->Cs = nullptr;
            st->Ce = nullptr;
            st->Y = nullptr;
            st->Ys = nullptr;
            DF_CUDA(cudaMalloc((void**)&st->Cs, sizeof(bf16) * st->S * (long long)ldy * np));
            DF_CUDA(cudaMalloc((void**)&st->Ce, sizeof(int) * ldy));
            DF_CUDA(cudaMalloc((void**)&st->Y, sizeof(float2) * (long long)h->naux * np * ldy));
            // (P, mu, i) slices for the mma.sync contraction, or (k block, mu, 64) with the last block padded
            DF_CUDA(cudaMalloc((void**)&st->Ys, sizeof(bf16) * st->S * np * ((long long)h->naux * ldy + 64)));
            st->ldy_cap = ldy;
        }
        // exponents per block: PB auxiliary rows (mma.sync layout) or an exact chunk of the contiguous
        // contraction index (tensor-core layout; the shortest chunk, S = SMAX, has the most blocks)
        const long long nblk = (h->naux + st->PB - 1) / st->PB;
        const long long nchk = ((long long)h->naux * ldy + exact_chunk<SMAX>() - 1) / exact_chunk<SMAX>();
        if (std::max(nblk, nchk) * np > st->ye_cap) {
            cudaFree(st->Ye);
            st->Ye = nullptr;
            DF_CUDA(cudaMalloc((void**)&st->Ye, sizeof(int) * std::max(nblk, nchk) * np));
            st->ye_cap = std::max(nblk, nchk) * np;
        }
        if (st->nsplit > st->kpart_cap) {
            cudaFree(st->Kpart);
            st->Kpart = nullptr;
            DF_CUDA(cudaMalloc((void**)&st->Kpart, sizeof(float2) * st->nsplit * np * np));
            st->kpart_cap = st->nsplit;
        }
        if (!st->err) {
            DF_CUDA(cudaMalloc((void**)&st->err, sizeof(int)));
            DF_CUDA(cudaMemsetAsync(st->err, 0, sizeof(int), h->stream));
        }
        // tcgen05 K: lower 128-tile pairs (fixed by np), split over exponent blocks to fill the GPU
        if (!st->tiles128) {
            const int nt128 = (int)((np + 127) / 128);
            st->npt = nt128 * 128;
            st->ntiles128 = nt128 * (nt128 + 1) / 2;
            std::vector<int2> t128;
            for (int I = 0; I < nt128; ++I)
                for (int J = 0; J <= I; ++J) t128.push_back(make_int2(I, J));
            DF_CUDA(cudaMalloc((void**)&st->tiles128, sizeof(int2) * t128.size()));
            DF_CUDA(cudaMemcpy(st->tiles128, t128.data(), sizeof(int2) * t128.size(), cudaMemcpyHostToDevice));
        }
        st->nsplit_tc = std::max(1, std::min((4 * 152 + 2 * st->ntiles128 - 1) / (2 * st->ntiles128), (int)nchk));
        st->ksplit_heur = st->nsplit_tc;
        if (st->nsplit_tc > st->kcap) {
            cudaFree(st->Kpart_tc);
            st->Kpart_tc = nullptr;
            DF_CUDA(cudaMalloc((void**)&st->Kpart_tc, sizeof(float2) * st->nsplit_tc * (long long)st->npt * st->npt));
            st->kcap = st->nsplit_tc;
        }
    }
    // synchronous callers clear the timeout flag per call; under the SCF driver it stays set once
    // raised and is read with the iteration's scalars
    } catch (...) {
        cudaStreamSynchronize(h->stream);   // nothing queued may still use the buffers freed here
        free_split(h);
        throw;
    }
    if (st->err && !h->tc_err_host) DF_CUDA(cudaMemsetAsync(st->err, 0, sizeof(int), h->stream));
    switch (slices) {
        case 2: run_split<2>(h, st, dC, nocc, dK, ev); break;
        case 3: run_split<3>(h, st, dC, nocc, dK, ev); break;
        case 4: run_split<4>(h, st, dC, nocc, dK, ev); break;
        default: run_split<5>(h, st, dC, nocc, dK, ev); break;
    }
    ev.mark(5, h->stream);
    if (st->err && h->tc_err_host) {
        DF_CUDA(cudaMemcpyAsync(h->tc_err_host, st->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    } else if (st->err) {
        // the tcgen05 kernels bound their waits and report expiry here
        int herr = 0;
        DF_CUDA(cudaMemcpyAsync(&herr, st->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        DF_CUDA(cudaStreamSynchronize(h->stream));
        if (herr) throw Error{DF_E_TIMEOUT, "tensor-core exchange kernel timed out waiting on a barrier"};
    }
    if (ev.on) {
        ev.sync(5);
        h->timings_ms[8] = ev.ms(0, 5);
        h->timings_ms[9] = ev.ms(1, 2);    // Y = B C (split)
        h->timings_ms[10] = ev.ms(3, 4);   // K contraction (split)
        h->timings_ms[11] = h->timings_ms[8] - h->timings_ms[9] - h->timings_ms[10];   // slicing, reduce
    }
}

double* split_y_buffer(df_handle* h, long long elems) {
    const SplitState* st = h->split;
    if (!st || !st->Y || (long long)h->naux * st->np * st->ldy_cap < elems) return nullptr;
    return reinterpret_cast<double*>(st->Y);
}

void split_clear_error(df_handle* h) {
    if (h->split && h->split->err) DF_CUDA(cudaMemsetAsync(h->split->err, 0, sizeof(int), h->stream));
}

}  // namespace dfhf
