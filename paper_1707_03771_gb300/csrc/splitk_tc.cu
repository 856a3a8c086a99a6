// Split-precision exchange on the 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
// Same arithmetic as split_k.cu (Ozaki slices, exact 512-element FP32 chunks, float-float drains), with
// the products issued as tcgen05.mma kind::f16 (BF16 x BF16 -> FP32 in tensor memory):
//   * one CTA owns an output tile of 128 rows x N columns; every Ozaki level L = s + t (0-based) has
//     its own FP32 accumulator of N columns in TMEM (S levels, S * N <= 512 columns);
//   * a producer thread streams K-steps of 64 elements with TMA (3-D tensor maps, 128-byte swizzle):
//     the S B slices of a K-step (N x 64 each) once into one of two resident buffers, and the S A
//     slices (128 x 64) through a ring of slots; every buffer is guarded by mbarriers;
//   * one thread issues the MMAs: for A slice s, the B slices t < S - s in wide MMAs (4 k16 steps
//     each), then commits the A slot back to the producer, and the B buffer after the K-step's last
//     A slice; at every chunk boundary it commits to the epilogue and waits until TMEM is free;
//   * four epilogue warps (one per 32 TMEM lanes) read the level sums with tcgen05.ld, scale them by the
//     exact power of two 2^{e_row + e_col - 7 (L + 2)} and add them into per-thread float-float rows.
// Every mbarrier wait is bounded by a clock budget; on expiry the kernel records DF_E_TIMEOUT in a flag,
// waits (with the full budget) for the copies and MMAs it has already issued, releases its tensor memory and
// returns.
//
// A third mode runs the metric whitening B = L^-1 A (paper eq. 1, third form) the same way with 7 slices:
// A operand = slices of L^-1 rows (one exponent per auxiliary row), B operand = slices of the
// transposed three-index columns (one exponent per pair column), K over the auxiliary index up to the
// end of the lower triangle, exact 448-element chunks (7 slices: a level sum is below 9 * 2^12 per
// term, 448 terms stay below 2^24), output in FP64.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "common.cuh"
#include "ozaki.cuh"

namespace dfhf {

namespace {

typedef __nv_bfloat16 bf16;

constexpr int TM = 128;            // output rows per CTA (TMEM lanes)
constexpr int KS = 64;             // K elements per pipeline step (one 128-byte swizzle row)
// pipeline steps per exact chunk: 12 (S = 3), 9 (S = 5), 7 (whitening, S = 7)
template <int S>
constexpr int chunk_steps() {
    return exact_chunk<S>() / KS;
}
// A-slice ring slots (one 128 x 64 slice each): 4, or 3 where that lets two CTAs share an SM
template <int S, int N>
constexpr int ring_slots() {
    return (S >= 7 && N <= 32) ? 3 : 4;
}
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz

// ------------------------------------------------------------------------------------------------
// PTX helpers
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded pipeline wait: false (and the error flag set) if the barrier did not complete within `budget`
// cycles (WAIT_CYCLES unless the host shortened it). The waits that drain copies and MMAs already issued,
// before the CTA leaves, always keep the full WAIT_CYCLES.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err, long long budget) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > budget || *(volatile int*)err) {
            atomicExch(err, DF_E_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// MN-major operand (the M index contiguous in shared memory, 128-byte swizzle): the tile is two 8 KB halves
// of 64 M-values each (one per TMA box), each half 8 K-rows of 128 bytes per 1024-byte atom. One stride
// field steps between the halves (along M), the other between 8-row atoms (along K).
constexpr unsigned MN_LBO = 8192;   // bytes between the two 64-wide M halves
constexpr unsigned MN_SBO = 1024;   // bytes between 8-row atoms along K
__device__ __forceinline__ uint64_t smem_desc_mn(const void* tile) {
    const unsigned a = smem_u32(tile);
    uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
    d |= (uint64_t)(MN_LBO >> 4) << 16;
    d |= (uint64_t)(MN_SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 bytes apart
__device__ __forceinline__ uint64_t smem_desc(const void* tile) {
    const unsigned a = smem_u32(tile);
    uint64_t d = (uint64_t)((a & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused with 128-byte swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                  // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                  // swizzle: 128 bytes
    return d;
}

// instruction descriptor: kind::f16, A and B BF16 (K-major), D FP32, M x N
__host__ __device__ constexpr unsigned instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, uint64_t a, uint64_t b, unsigned idesc, unsigned accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float pow2f(int e) { return e < -126 ? 0.f : __int_as_float((127 + min(e, 127)) << 23); }


__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (v - bb);
    hi = s;
    lo += err;
}

// ------------------------------------------------------------------------------------------------
// Work description. MODE 0 (Y = B C): CTA = (P, mu-tile, n-tile); K runs over nu (np), exponents
// constant (row: Be[P][mu], column: Ce[i]). MODE 3 (Y = B C from the packed slices): B_P is stored as its
// lower 128 x 128 tiles only, Bs[s][P][t][128][128] with t = I (I + 1) / 2 + J for I >= J (diagonal tiles
// whole), one exponent per P (Be[P]); K-step blocks nu of J > I come from the stored tile (J, I) read as an
// MN-major (transposed) operand. MODE 1 (K = sum Y Y^T): CTA = (split, lower tile pair,
// column part), the split slowest so that the CTAs resident together stream the same range of the
// contraction through L2; K runs over the contiguous index k = P ldy + i of the Y slices, stored tile-major
// as Ys[s][k / 64][mu][k % 64] (one TMA box is 16 KB of contiguous memory; no padding between auxiliary
// rows), one exact chunk per block of consecutive k with its own exponents Ye[block][mu], Ye[block][nu].
// ------------------------------------------------------------------------------------------------
struct TcArgs {
    int mode;
    int naux, np, ldy, PB, nsplit;
    long long KL;            // MODE 1: naux * ldy, the length of the contraction
    int nkb;                 // MODE 1: 64-wide blocks of the contraction, ceil(KL / 64)
    int ntiles;              // MODE 1: lower 128-tile pairs
    const int* row_e;        // MODE 0: Be [naux][np]; MODE 1: Ye [nchunk][np]
    const int* col_e;        // MODE 0: Ce [ldy]
    const int2* tiles;       // MODE 1: lower 128-tile pairs
    float2* out;             // MODE 0: Y [naux][np][ldy]; MODE 1: Kpart [nsplit][npt][npt]
    int npt;                 // MODE 1: padded dimension of Kpart (multiple of 128)
    int* err;
    // MODE 2 (whitening): rows = naux (np is set to naux), ncols pair columns of this chunk,
    // row_e = L^-1 row exponents, col_e = column exponents, output FP64 rows of stride ldo
    int ncols;
    double* outd;
    long long ldo;
    long long wait_cycles;   // budget of the pipeline waits (WAIT_CYCLES by default)
    int nB;                  // MODE 3: 128-row blocks of the packed tiles (np padded to 128 nB)
};

template <int S, int N, int MODE>
__global__ void __launch_bounds__(192, 1) ozaki_tc_kernel(const __grid_constant__ CUtensorMap mapA,
                                                          const __grid_constant__ CUtensorMap mapB, TcArgs args) {
    constexpr int A_BYTES = TM * KS * 2;          // 16 KB
    constexpr int B_BYTES = N * KS * 2;           // a multiple of 1024 (N a multiple of 16)
    constexpr int BSET = S * B_BYTES;             // every B slice of one K-step
    constexpr int NA = ring_slots<S, N>();
    constexpr int NCOLS = S * N <= 32 ? 32 : (S * N <= 64 ? 64 : (S * N <= 128 ? 128 : (S * N <= 256 ? 256 : 512)));
    static_assert(S * N <= 512, "TMEM holds at most 512 accumulator columns");
    constexpr int MMA_SLICES = 256 / N;            // B slices per MMA (M = 128 allows N <= 256)
    static_assert(N % 16 == 0 && N <= 256, "MMA width");

    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* bbuf = smem + NA * A_BYTES;    // two B sets
    uint64_t* a_full = (uint64_t*)(bbuf + 2 * BSET);
    uint64_t* a_empty = a_full + NA;
    uint64_t* b_full = a_empty + NA;
    uint64_t* b_empty = b_full + 2;
    uint64_t* acc_full = b_empty + 2;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* mma_done = acc_empty + 1;
    unsigned* tmem_slot = (unsigned*)(mma_done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* err = args.err;
    const long long wait = args.wait_cycles;

    // ---- work decode -------------------------------------------------------------------------
    int P = 0, m0 = 0, n0 = 0, split = 0;
    int2 IJ = make_int2(0, 0);
    int ksteps = 0;
    int p0 = 0, kpp = 0;   // MODE 1: first chunk and first K-step of the split
    if (MODE == 0 || MODE == 3) {
        const int mt = MODE == 3 ? args.nB : (args.np + TM - 1) / TM;
        const int nt = args.ldy / N;
        int b = blockIdx.x;
        const int ntile = b % nt;
        b /= nt;
        m0 = (b % mt) * TM;
        P = b / mt;
        n0 = ntile * N;
        ksteps = MODE == 3 ? 2 * args.nB : args.np / KS;
    } else if (MODE == 2) {
        const int ntn = args.ncols / N;
        m0 = (blockIdx.x / ntn) * TM;             // row-tile major: the L^-1 tile is shared in L2
        n0 = (blockIdx.x % ntn) * N;
        ksteps = (min(args.naux, m0 + TM) + KS - 1) / KS;   // L^-1 is lower triangular
    } else {
        const int halves = TM / N;
        int b = blockIdx.x;
        const int h = b % halves;
        b /= halves;
        IJ = args.tiles[b % args.ntiles];
        split = b / args.ntiles;
        m0 = IJ.x * TM;
        n0 = IJ.y * TM + h * N;
        constexpr int CH = exact_chunk<S>();
        const long long nchk = (args.KL + CH - 1) / CH;
        const long long c0 = nchk * split / args.nsplit, c1 = nchk * (split + 1) / args.nsplit;
        p0 = (int)c0;                                              // first chunk of this split
        const long long k0 = c0 * CH, k1 = min(args.KL, c1 * CH);
        kpp = (int)(k0 / KS);                                      // first K-step (chunks are K-step aligned)
        ksteps = (int)((k1 - k0 + KS - 1) / KS);
    }

    // ---- set-up: barriers (thread 0), tensor memory (warp 0) ------------------------------------
    if (threadIdx.x == 0) {
        for (int i = 0; i < NA; ++i) {
            mbar_init(&a_full[i], 1);
            mbar_init(&a_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&b_full[i], 1);
            mbar_init(&b_empty[i], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 128);
        mbar_init(mma_done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = *tmem_slot;

    // chunk index of K-step ks (every mode: the exact chunk of S slices)
    auto chunk_of = [&](int ks) { return ks / chunk_steps<S>(); };
    const int nchunks = ksteps > 0 ? chunk_of(ksteps - 1) + 1 : 0;

    if (warp == 4) {
        // ---------------------------------- producer ------------------------------------------
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];\n" ::"l"((unsigned long long)&mapA) : "memory");
            asm volatile("prefetch.tensormap [%0];\n" ::"l"((unsigned long long)&mapB) : "memory");
            int a_issued = 0, b_issued = 0;
            for (int ks = 0; ks < ksteps; ++ks) {
                // x: the contraction coordinate of this K-step; MODE 1 reads the tile-major slices
                // [s][k block][row][64] at x = 0 and z = s nkb + the split's K-step
                const int kx = MODE == 1 ? 0 : ks * KS;
                const int kb = kpp + ks;
                const int bs = ks & 1;
                if (!mbar_wait(&b_empty[bs], ((ks >> 1) & 1) ^ 1, err, wait)) break;
                mbar_expect_tx(&b_full[bs], BSET);
                for (int t = 0; t < S; ++t)
                    tma_load_3d(bbuf + bs * BSET + t * B_BYTES, &mapB, kx, n0, MODE == 1 ? t * args.nkb + kb : t,
                                &b_full[bs]);
                ++b_issued;
                bool ok = true;
                for (int s = 0; s < S; ++s) {
                    const int it = ks * S + s, slot = it % NA;
                    if (!mbar_wait(&a_empty[slot], ((it / NA) & 1) ^ 1, err, wait)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&a_full[slot], A_BYTES);
                    const int za = (MODE == 0 || MODE == 3) ? s * args.naux + P : (MODE == 1 ? s * args.nkb + kb : s);
                    if (MODE == 3) {
                        // two 64-row boxes of one stored tile: rows mu of tile (I, J) at columns nu of this
                        // K-step (K-major), or, above the diagonal, rows nu of tile (J, I) (MN-major halves)
                        const int I = m0 / TM, J = ks >> 1, half = ks & 1;
                        unsigned char* dst = smem + slot * A_BYTES;
                        if (I >= J) {
                            const int y0 = (I * (I + 1) / 2 + J) * TM;
                            tma_load_3d(dst, &mapA, half * KS, y0, za, &a_full[slot]);
                            tma_load_3d(dst + A_BYTES / 2, &mapA, half * KS, y0 + KS, za, &a_full[slot]);
                        } else {
                            const int y0 = (J * (J + 1) / 2 + I) * TM + half * KS;
                            tma_load_3d(dst, &mapA, 0, y0, za, &a_full[slot]);
                            tma_load_3d(dst + A_BYTES / 2, &mapA, KS, y0, za, &a_full[slot]);
                        }
                    } else {
                        tma_load_3d(smem + slot * A_BYTES, &mapA, kx, m0, za, &a_full[slot]);
                    }
                    ++a_issued;
                }
                if (!ok) break;
            }
            // copies in flight complete before the kernel may leave: wait (bounded) for the last ones of every
            // slot. After a normal run the MMA issuer has consumed them all and these waits return at once;
            // after a timeout (here or in the issuer, which may give up while this thread has finished its
            // loop) they keep the CTA until its copies have landed.
            for (int it = max(0, a_issued - NA); it < a_issued; ++it) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&a_full[it % NA], (it / NA) & 1) && clock64() - t0 < WAIT_CYCLES) {
                }
            }
            for (int k = max(0, b_issued - 2); k < b_issued; ++k) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&b_full[k & 1], (k >> 1) & 1) && clock64() - t0 < WAIT_CYCLES) {
                }
            }
        }
    } else if (warp == 5) {
        // ---------------------------------- MMA issuer ----------------------------------------
        if (lane == 0) {
            int chunk = 0;
            bool ok = true;
            for (int ks = 0; ks < ksteps && ok; ++ks) {
                const int c = chunk_of(ks);
                if (c != chunk) {                 // new chunk: hand the finished sums to the epilogue
                    mma_commit(acc_full);
                    ok = mbar_wait(acc_empty, (chunk & 1), err, wait);
                    fence_after();
                    chunk = c;
                    if (!ok) break;
                }
                const int bs = ks & 1;
                if (!mbar_wait(&b_full[bs], (ks >> 1) & 1, err, wait)) {
                    ok = false;
                    break;
                }
                fence_after();
                const bool first_in_chunk = ks == 0 || chunk_of(ks - 1) != c;
                unsigned char* bset = bbuf + bs * BSET;
                const bool mn = MODE == 3 && m0 / TM < (ks >> 1);   // A read transposed from the stored tile
                const unsigned amaj = mn ? (1u << 15) : 0u;
                for (int s = 0; s < S; ++s) {
                    const int it = ks * S + s, slot = it % NA;
                    if (!mbar_wait(&a_full[slot], (it / NA) & 1, err, wait)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    // the B slices t < S - s are consecutive N-row tiles in shared memory and their levels
                    // s + t consecutive N-column accumulators in TMEM, so up to 256 / N of them form one
                    // MMA of width cnt * N (one read of the A tile per MMA instead of one per slice)
#pragma unroll
                    for (int k = 0; k < KS / 16; ++k) {
                        // K-major: +32 B per k16; MN-major: +2 atoms of 8 K-rows (2048 B) per k16
                        const uint64_t ad = mn ? smem_desc_mn(smem + slot * A_BYTES + k * 2048)
                                               : smem_desc(smem + slot * A_BYTES) + (uint64_t)(k * 2);
                        for (int t = 0; t < S - s; t += MMA_SLICES) {
                            const int cnt = min(MMA_SLICES, S - s - t);
                            const uint64_t bd = smem_desc(bset + t * B_BYTES) + (uint64_t)(k * 2);
                            mma_bf16(tmem + (unsigned)((s + t) * N), ad, bd, instr_desc(TM, cnt * N) | amaj,
                                     (first_in_chunk && s == 0 && k == 0) ? 0u : 1u);
                        }
                    }
                    mma_commit(&a_empty[slot]);
                }
                if (ok) mma_commit(&b_empty[bs]);
            }
            if (ok && ksteps > 0) mma_commit(acc_full);
            // every MMA this thread issued has completed before tensor memory is released
            mma_commit(mma_done);
            const long long t0 = clock64();
            while (!mbar_try_wait(mma_done, 0) && clock64() - t0 < WAIT_CYCLES) {
            }
        }
    } else {
        // ---------------------------------- epilogue (warps 0-3) ------------------------------
        // MODE 0 and 2: exponents are the same for every chunk, so chunk sums are accumulated with the
        // level factor 2^{-7(L+2)} only and the row/column powers of two are applied once at the end.
        const int row = warp * 32 + lane;               // TMEM lane = tile row
        const int grow = m0 + row;
        float hi[N], lo[N];
#pragma unroll
        for (int c = 0; c < N; ++c) hi[c] = lo[c] = 0.f;
        const unsigned lane_base = tmem + ((unsigned)(warp * 32) << 16);
        for (int ch = 0; ch < nchunks; ++ch) {
            int erow = 0;
            long long blk = 0;
            if (MODE == 1) {
                blk = p0 + ch;
                erow = (grow < args.np) ? args.row_e[blk * args.np + grow] : 0;
            }
            if (!mbar_wait(acc_full, ch & 1, err, wait)) break;
            fence_after();
            // per element the levels are added in descending order; column exponents (MODE 1) are read
            // per 16-column group to keep them out of the register file
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 16) {
                int ce[16];
                if (MODE == 1) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        ce[j] = (n0 + c0 + j < args.np) ? __ldg(args.row_e + blk * args.np + n0 + c0 + j) : 0;
                }
#pragma unroll 1
                for (int L = S - 1; L >= 0; --L) {
                    const float lev = pow2f(-7 * (L + 2));
                    float v[16];
                    tmem_ld16(lane_base + (unsigned)(L * N + c0), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float sc = (MODE == 1) ? pow2f(erow + ce[j] - 7 * (L + 2)) : lev;
                        two_sum_acc(hi[c0 + j], lo[c0 + j], v[j] * sc);
                    }
                }
            }
            fence_before();
            mbar_arrive(acc_empty);
        }
        // output
        if (!*(volatile int*)err && grow < args.np) {
            if (MODE == 2) {
                const int er = args.row_e[grow];
                double* o = args.outd + (long long)grow * args.ldo + n0;
#pragma unroll
                for (int c = 0; c < N; ++c)
                    o[c] = scale_pow2((double)hi[c] + (double)lo[c], er + __ldg(args.col_e + n0 + c));
            } else if (MODE == 0 || MODE == 3) {
                const int er = MODE == 3 ? args.row_e[P] : args.row_e[(long long)P * args.np + grow];
                float2* o = args.out + ((long long)P * args.np + grow) * args.ldy + n0;
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    const float f = pow2f(er + __ldg(args.col_e + n0 + c));
                    o[c] = make_float2(hi[c] * f, lo[c] * f);
                }
            } else {
                float2* o = args.out + ((long long)split * args.npt + grow) * args.npt + n0;
#pragma unroll
                for (int c = 0; c < N; ++c) o[c] = make_float2(hi[c], lo[c]);
            }
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOLS));
}

template <int S, int N>
size_t tc_smem_bytes() {
    return (size_t)ring_slots<S, N>() * TM * KS * 2 + 2 * (size_t)S * N * KS * 2 + 1024 + 256;
}

// ------------------------------------------------------------------------------------------------
// tensor maps through the driver entry point (no link-time dependence on libcuda)
// ------------------------------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::mutex mu;
    static EncodeTiledFn fn = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        DF_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) throw Error{DF_E_CUDA, "cuTensorMapEncodeTiled unavailable"};
        fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 3-D BF16 tensor [d2][d1][d0] (d0 contiguous) with box {64, rows, 1}, 128-byte swizzle, zero fill
CUtensorMap make_map(const bf16* base, unsigned long long d0, unsigned long long d1, unsigned long long d2,
                     unsigned rows) {
    CUtensorMap m;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {d0 * 2, d0 * d1 * 2};
    const cuuint32_t box[3] = {(cuuint32_t)KS, rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error{DF_E_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r)};
    return m;
}

// Budget of the kernels' pipeline waits: WAIT_CYCLES, or DFHF_TC_WAIT_CYCLES (a test knob that makes the
// waits run out, to exercise the DF_E_TIMEOUT path; the drains of work already issued keep WAIT_CYCLES)
long long pipeline_wait_cycles() {
    const char* v = std::getenv("DFHF_TC_WAIT_CYCLES");
    const long long c = v ? std::atoll(v) : 0;
    return (c > 0 && c < WAIT_CYCLES) ? c : WAIT_CYCLES;
}

template <int S, int N, int MODE>
void launch_tc(cudaStream_t s, const CUtensorMap& a, const CUtensorMap& b, const TcArgs& args_in, unsigned grid) {
    const size_t smem = tc_smem_bytes<S, N>();
    TcArgs args = args_in;
    args.wait_cycles = pipeline_wait_cycles();
    DF_CUDA(cudaFuncSetAttribute(ozaki_tc_kernel<S, N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ozaki_tc_kernel<S, N, MODE><<<grid, 192, smem, s>>>(a, b, args);
    DF_CHECK_LAUNCH();
}

// K[mu][nu] (n x n, FP64) = sum over splits of the float pairs, read from the computed lower 128-tiles
__global__ void k_tc_reduce_kernel(const float2* __restrict__ Kpart, int nsplit, int npt, int n, double* __restrict__ K) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    int a = (int)(idx / n), b = (int)(idx % n);
    if (a / TM < b / TM) {
        const int t = a;
        a = b;
        b = t;
    }
    double s = 0.0;
    for (int q = 0; q < nsplit; ++q) {
        const float2 v = Kpart[((long long)q * npt + a) * npt + b];
        s += (double)v.x + (double)v.y;
    }
    K[idx] = s;
}

}  // namespace

void k_tc_reduce(cudaStream_t s, const float2* Kpart, int nsplit, int npt, int n, double* K) {
    const long long nn = (long long)n * n;
    k_tc_reduce_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(Kpart, nsplit, npt, n, K);
    DF_CHECK_LAUNCH();
}

// Y[P][mu][i] (float pairs) = B_P C from the slices Bs [S][naux][np][np], Cs [S][ldy][np]; CTA tiles
// of 128 rows x N columns, N in {32, 64, 80} dividing ldy (chosen by the autotuner)
template <int S, int N>
void y_tc_launch(cudaStream_t s, const CUtensorMap& ma, const bf16* Cs, int np, int ldy, const TcArgs& a, int naux) {
    const CUtensorMap mb = make_map(Cs, np, ldy, S, N);
    const unsigned mt = (np + TM - 1) / TM;
    launch_tc<S, N, 0>(s, ma, mb, a, (unsigned)naux * mt * (ldy / N));
}

void y_split_tc(cudaStream_t s, int S, int N, const bf16* Bs, const int* Be, const bf16* Cs, const int* Ce, int naux,
                int np, int ldy, float2* Y, int* err) {
    if (ldy % N) throw Error{DF_E_ARG, "tensor-core split Y: tile width must divide the occupied width"};
    TcArgs a{};
    a.mode = 0;
    a.naux = naux;
    a.np = np;
    a.ldy = ldy;
    a.row_e = Be;
    a.col_e = Ce;
    a.out = Y;
    a.err = err;
    const CUtensorMap ma = make_map(Bs, np, np, (unsigned long long)S * naux, TM);
    if (S == 3 && N == 80) y_tc_launch<3, 80>(s, ma, Cs, np, ldy, a, naux);
    else if (S == 5 && N == 80) y_tc_launch<5, 80>(s, ma, Cs, np, ldy, a, naux);
    else if (S == 3 && N == 64) y_tc_launch<3, 64>(s, ma, Cs, np, ldy, a, naux);
    else if (S == 5 && N == 64) y_tc_launch<5, 64>(s, ma, Cs, np, ldy, a, naux);
    else if (S == 3 && N == 32) y_tc_launch<3, 32>(s, ma, Cs, np, ldy, a, naux);
    else if (S == 5 && N == 32) y_tc_launch<5, 32>(s, ma, Cs, np, ldy, a, naux);
    else throw Error{DF_E_ARG, "tensor-core split Y supports 3 or 5 slices and tile widths 32, 64, 80"};
}

// Y from the packed slices Bs [S][naux][nB (nB + 1) / 2][128][128] (lower 128-tiles, one exponent Be[P]
// per auxiliary row): tile widths as y_split_tc
template <int S, int N>
void y_tc_packed_launch(cudaStream_t s, const CUtensorMap& ma, const bf16* Cs, int np, int ldy, const TcArgs& a,
                        int naux, int nB) {
    const CUtensorMap mb = make_map(Cs, np, ldy, S, N);
    launch_tc<S, N, 3>(s, ma, mb, a, (unsigned)naux * nB * (ldy / N));
}

// naux rows are computed; the slices of row P sit at z = s * zrows + P (zrows >= naux: the buffer's rows)
void y_split_tc_packed(cudaStream_t s, int S, int N, const bf16* Bs, const int* Be, const bf16* Cs, const int* Ce,
                       int naux, int zrows, int np, int nB, int ldy, float2* Y, int* err) {
    if (ldy % N) throw Error{DF_E_ARG, "tensor-core split Y: tile width must divide the occupied width"};
    if (np > nB * TM || np % KS) throw Error{DF_E_ARG, "internal: packed tiles do not cover the padded size"};
    if (zrows < naux) throw Error{DF_E_ARG, "internal: slice buffer smaller than the rows computed"};
    TcArgs a{};
    a.mode = 3;
    a.naux = zrows;
    a.np = np;
    a.ldy = ldy;
    a.nB = nB;
    a.row_e = Be;
    a.col_e = Ce;
    a.out = Y;
    a.err = err;
    const unsigned long long ntile = (unsigned long long)nB * (nB + 1) / 2;
    const CUtensorMap ma = make_map(Bs, TM, ntile * TM, (unsigned long long)S * zrows, KS);
    if (S == 3 && N == 80) y_tc_packed_launch<3, 80>(s, ma, Cs, np, ldy, a, naux, nB);
    else if (S == 5 && N == 80) y_tc_packed_launch<5, 80>(s, ma, Cs, np, ldy, a, naux, nB);
    else if (S == 3 && N == 64) y_tc_packed_launch<3, 64>(s, ma, Cs, np, ldy, a, naux, nB);
    else if (S == 5 && N == 64) y_tc_packed_launch<5, 64>(s, ma, Cs, np, ldy, a, naux, nB);
    else if (S == 3 && N == 32) y_tc_packed_launch<3, 32>(s, ma, Cs, np, ldy, a, naux, nB);
    else if (S == 5 && N == 32) y_tc_packed_launch<5, 32>(s, ma, Cs, np, ldy, a, naux, nB);
    else throw Error{DF_E_ARG, "tensor-core split Y supports 3 or 5 slices and tile widths 32, 64, 80"};
}

// B[P][c] = sum_Q L^-1[P][Q] A[Q][c] for the ncols columns of one chunk, from the 7 slices
// Ls [7][naux][kp] (row exponents eL) and At [7][ncols][kp] (column exponents eA); rows of `out` have
// stride ldo. kp is naux padded to a multiple of 64 (zero slices beyond naux), ncols a multiple of 64.
template <int N>
void whiten_tc_n(cudaStream_t s, const bf16* Ls, const int* eL, const bf16* At, const int* eA, int naux, int kp,
                 int ncols, double* out, long long ldo, int* err) {
    constexpr int S = 7;
    if (kp % KS || ncols % N) throw Error{DF_E_ARG, "internal: whitening operands not padded to 64"};
    TcArgs a{};
    a.mode = 2;
    a.naux = naux;
    a.np = naux;
    a.row_e = eL;
    a.col_e = eA;
    a.err = err;
    a.ncols = ncols;
    a.outd = out;
    a.ldo = ldo;
    const CUtensorMap ma = make_map(Ls, kp, naux, S, TM);
    const CUtensorMap mb = make_map(At, kp, ncols, S, N);
    const unsigned grid = (unsigned)((naux + TM - 1) / TM) * (unsigned)(ncols / N);
    launch_tc<S, N, 2>(s, ma, mb, a, grid);
}

// N: output tile width, 64 or 32 (32: two CTAs per SM)
void whiten_tc(cudaStream_t s, int N, const bf16* Ls, const int* eL, const bf16* At, const int* eA, int naux, int kp,
               int ncols, double* out, long long ldo, int* err) {
    if (N == 64) whiten_tc_n<64>(s, Ls, eL, At, eA, naux, kp, ncols, out, ldo, err);
    else if (N == 32) whiten_tc_n<32>(s, Ls, eL, At, eA, naux, kp, ncols, out, ldo, err);
    else throw Error{DF_E_ARG, "tensor-core whitening supports tile widths 32 and 64"};
}

// K partial sums over lower 128-tile pairs: Kpart [nsplit][npt][npt] (float pairs), from the Y slices
// Ys [S][KL / 64][np][64] (KL = naux ldy over the contraction index k = P ldy + i, tile-major) with exponents
// Ye [chunk][np]
template <int N>
void k_split_tc_n(cudaStream_t s, int S, const bf16* Ys, const int* Ye, int naux, int np, int ldy, int nsplit,
                  const int2* tiles128, int ntiles, float2* Kpart, int npt, int* err) {
    TcArgs a{};
    a.mode = 1;
    a.naux = naux;
    a.np = np;
    a.ldy = ldy;
    a.KL = (long long)naux * ldy;
    a.nkb = (int)((a.KL + KS - 1) / KS);
    a.ntiles = ntiles;
    a.nsplit = nsplit;
    a.row_e = Ye;
    a.tiles = tiles128;
    a.out = Kpart;
    a.npt = npt;
    a.err = err;
    const CUtensorMap ma = make_map(Ys, KS, np, (unsigned long long)S * a.nkb, TM);
    const CUtensorMap mb = make_map(Ys, KS, np, (unsigned long long)S * a.nkb, N);
    const unsigned grid = (unsigned)ntiles * nsplit * (TM / N);
    switch (S) {
        case 3: launch_tc<3, N, 1>(s, ma, mb, a, grid); break;
        case 5: launch_tc<5, N, 1>(s, ma, mb, a, grid); break;
        default: throw Error{DF_E_ARG, "tensor-core split K supports 3 or 5 slices"};
    }
}

// N: width of the column half-tiles of each 128 x 128 output tile, 64 or 32
void k_split_tc(cudaStream_t s, int S, int N, const bf16* Ys, const int* Ye, int naux, int np, int ldy, int nsplit,
                const int2* tiles128, int ntiles, float2* Kpart, int npt, int* err) {
    if (N == 64) k_split_tc_n<64>(s, S, Ys, Ye, naux, np, ldy, nsplit, tiles128, ntiles, Kpart, npt, err);
    else if (N == 32) k_split_tc_n<32>(s, S, Ys, Ye, naux, np, ldy, nsplit, tiles128, ntiles, Kpart, npt, err);
    else throw Error{DF_E_ARG, "tensor-core split K supports tile widths 32 and 64"};
}

}  // namespace dfhf
