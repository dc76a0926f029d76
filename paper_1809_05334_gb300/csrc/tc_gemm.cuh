// Complex FP32 products C <- beta C + A B (K <= 512) of the Gauss-Jordan
// inversion of the domain blocks of Eq. (6), on the 5th-generation tensor
// cores (tcgen05, kind::f16 with FP16 operands and FP32 accumulators in tensor
// memory), with every operand moved by TMA.  FP16 keeps the 10-bit mantissa
// of TF32 at half the operand bytes and twice the rate; its range is handled
// by a power-of-two scale per packed operand (its largest entry brought to
// [2^13, 2^14)), undone in the epilogue.
//
// A complex product is one real product of the real views:
//   C_rv (M x 2N) += A_rv (M x 2K) * Bt (2K x 2N)
// where the real view of a row-major complex matrix interleaves (re, im) and
// Bt is the 2x2 real expansion of B (times a sign).  Pack kernels write (FP16)
//   Ap [mp][2 KP]    row r: K complex entries of the r-th row of A
//   Bp [2 np][2 KP]  rows 2j, 2j+1: s (Re b, -Im b), s (Im b, Re b), b = B[k][j]
// so that both operands are K-major and TMA-loadable (zero padded to 128-row
// tiles and to KP = 1024; a product reads the first kchunks x 64 real K).  Rows and columns of C are addressed through
// skip maps (index i < at ? i : i + skip), so a product can cover the trailing
// rows/columns around a pivot block, the pivot columns alone, or all rows.
//
// k_tc_update is persistent (one CTA per SM, tiles of 128 x 128 complex taken
// round-robin in column-by-column order) and warp-specialised:
//   warp 0   TMA producer of the A/B chunks (64 real K each) into a 3-stage ring
//   warp 1   tensor-memory allocation (512 columns = two 128 x 256 FP32
//            accumulators) and the MMA issuer (M=128, N=256, K=16)
//   warp 2   TMA producer of C, in 128-row x 32-float chunks, into a 4-slot ring
//   warps 4-7  epilogue: tcgen05.ld of the accumulator (lane = row), add to the
//            staged C chunk, TMA store of each warp's 32 rows
// so the C traffic of one tile overlaps the MMAs of the next.  Every mbarrier
// wait has an iteration limit; on timeout the role records an error, stops,
// waits (bounded) for the copies and MMAs it issued, and the CTA still frees
// its tensor memory.  Warp-level decisions are made uniform with a vote, and no
// barrier other than the final __syncthreads spans several warps.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace vie {

constexpr int TC_TM = 128;                        // complex rows per tile
constexpr int TC_TN = 128;                        // complex columns per tile (256 real)
constexpr int TC_KP = 1024;                       // complex K of the packed operands (zero padded)
constexpr int TC_KCHUNK = 64;                     // real K (FP16) per stage: one 128-byte swizzle row
constexpr int TC_CCHUNK = 2 * TC_TN / 32;         // 8 chunks of 32 floats across a C tile
constexpr int TC_A_BYTES = TC_TM * 128;           // 16 KB
constexpr int TC_B_BYTES = 2 * TC_TN * 128;       // 32 KB
constexpr int TC_C_BYTES = TC_TM * 128;           // 16 KB: 128 rows x 32 floats of C
constexpr int TC_STAGES = 3;
constexpr int TC_CSLOTS = 4;
constexpr int TC_BAR_BYTES = 256;
constexpr int TC_SMEM = 1024 + TC_STAGES * (TC_A_BYTES + TC_B_BYTES) + TC_CSLOTS * TC_C_BYTES + TC_BAR_BYTES;
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr long long TC_WAIT_LIMIT = 20000000;     // polls of one wait (tens of ms)
constexpr int TC_THREADS = 256;
constexpr int TC_PACK_ROW = 2 * TC_KP;            // FP16 entries per packed row (4 KB)

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 1024-byte atom stride
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused for K-major swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: 8-row atoms
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)2 << 61;                           // SWIZZLE_128B
    return d;
}

// instruction descriptor: D f32, A and B f16, K-major, N = 256, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

// Exponent x of the power-of-two scale 2^x that brings a packed operand's
// largest entry (given as the bits of a non-negative float) into [2^13, 2^14):
// x = 13 - e for amax = 1.f.. x 2^e, read from the exponent field; 0 for a zero
// or non-finite amax; clamped to [-120, 120] (subnormal amax take 120).
__device__ __forceinline__ int tc_shift(unsigned amax_bits) {
    const int be = (int)((amax_bits >> 23) & 0xffu);
    if (amax_bits == 0u || be == 0xff) return 0;
    const int x = 13 - (be - 127);
    return x < -120 ? -120 : (x > 120 ? 120 : x);
}
__device__ __forceinline__ float tc_pow2(int x) { return __int_as_float((127 + x) << 23); }   // |x| <= 126


// bounded wait on an mbarrier phase; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, long long limit = TC_WAIT_LIMIT) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(mbar))
        : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(src)), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(mbar)) : "memory");
}

// One operand panel of a product, as the pack kernels read it: mode A (k_tc_pack_a)
// rows r < n1 at row(r) = r < at ? r : r + skip, columns c0 .. c0 + w; mode B
// (k_tc_pack_b) rows c0 .. c0 + w, columns j < n1 at col(j) = j < at ? j : j + skip.
struct TcPanel {
    int n1, c0, w, at, skip;
};

// Largest |Re|, |Im| of panel pa (blockIdx.y = 0, mode A) and pb (1, mode B),
// atomicMax-ed as float bits into out[blockIdx.y] (zeroed by the caller).
__global__ void __launch_bounds__(256) k_tc_absmax(const float *__restrict__ A, size_t ld, TcPanel pa, TcPanel pb,
                                                   unsigned *out) {
    const bool mb = blockIdx.y != 0;
    const TcPanel p = mb ? pb : pa;
    const int tot = p.n1 * p.w;
    float mx = 0.f;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
        size_t idx;
        if (!mb) {   // row r (mapped), column c0 + k: consecutive e along a row
            const int r = e / p.w, k = e - r * p.w;
            idx = (size_t)(r < p.at ? r : r + p.skip) * ld + p.c0 + k;
        } else {     // row c0 + k, column j (mapped): consecutive e along a row
            const int k = e / p.n1, j = e - k * p.n1;
            idx = (size_t)(p.c0 + k) * ld + (j < p.at ? j : j + p.skip);
        }
        const float2 v = *reinterpret_cast<const float2 *>(A + 2 * idx);
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + blockIdx.y, __float_as_uint(mx));
}

// Ap[r][2k..2k+1] = s A[row(r)][col0 + k] for r < rows, k < w, with
// row(r) = r < at ? r : r + skip; zero elsewhere up to mp rows and kp columns
// (the K chunks a product reads); s from *amax.
__global__ void __launch_bounds__(256) k_tc_pack_a(const float *__restrict__ A, size_t ld, int rows, int col0, int w,
                                                   int at, int skip, int mp, int kp, const unsigned *__restrict__ amax,
                                                   __half *__restrict__ Ap) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)mp * kp) return;
    const int r = (int)(e / kp), k = (int)(e % kp);
    float2 v = make_float2(0.f, 0.f);
    if (r < rows && k < w) {
        const int gr = r < at ? r : r + skip;
        v = *reinterpret_cast<const float2 *>(A + 2 * ((size_t)gr * ld + col0 + k));
    }
    const float s = tc_pow2(tc_shift(*amax));
    *reinterpret_cast<__half2 *>(Ap + (size_t)r * TC_PACK_ROW + 2 * k) = __floats2half2_rn(s * v.x, s * v.y);
}

// The sign- and power-of-two-scaled real expansion of B[k][j] = A[row0 + k][col(j)]
// (k < w, j < cols, col(j) = j < at ? j : j + skip), K-major:
//   Bp[2j][2k..] = sgn s (Re b, -Im b),  Bp[2j+1][2k..] = sgn s (Im b, Re b)
// through a 32 x 32 shared-memory transpose (coalesced on both sides); rows up
// to 2 * 32 * gridDim.x and K up to 32 * gridDim.y are written (zero beyond
// cols and w).
__global__ void __launch_bounds__(256) k_tc_pack_b(const float *__restrict__ A, size_t ld, int cols, int row0, int w,
                                                   int at, int skip, float sgn, const unsigned *__restrict__ amax,
                                                   __half *__restrict__ Bp) {
    __shared__ float2 t[32][33];
    const int j0 = blockIdx.x * 32, kb = blockIdx.y * 32;
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
        const int kk = idx / 32, jj = idx % 32;
        const int j = j0 + jj, k = kb + kk;
        float2 v = make_float2(0.f, 0.f);
        if (j < cols && k < w) {
            const int gc = j < at ? j : j + skip;
            v = *reinterpret_cast<const float2 *>(A + 2 * ((size_t)(row0 + k) * ld + gc));
        }
        t[kk][jj] = v;
    }
    __syncthreads();
    const float g = sgn * tc_pow2(tc_shift(*amax));
    for (int idx = threadIdx.x; idx < 32 * 32; idx += blockDim.x) {
        const int jj = idx / 32, kk = idx % 32;
        const float2 v = t[kk][jj];
        const size_t j = (size_t)(j0 + jj), k = (size_t)(kb + kk);
        *reinterpret_cast<__half2 *>(Bp + (2 * j) * TC_PACK_ROW + 2 * k) = __floats2half2_rn(g * v.x, -g * v.y);
        *reinterpret_cast<__half2 *>(Bp + (2 * j + 1) * TC_PACK_ROW + 2 * k) = __floats2half2_rn(g * v.y, g * v.x);
    }
}

// Index maps and scaling of one product: C rows r < mrows at row(r) =
// r < rat ? r : r + rskip, columns c < ncols at col(c) = c < cat ? c : c + cskip
// (rat, cat multiples of 128 or beyond the extent, so no tile straddles a
// skip); beta = 0 on every tile if beta0_all, else on the tile rows
// [beta0_lo, beta0_lo + beta0_n).
// only_n > 0 restricts the product to the tile columns [only_lo, only_lo +
// only_n); skip_n > 0 leaves the tile columns [skip_lo, skip_lo + skip_n) out
// (the two parts of a split product).  kchunks: chunks of 64 real K read.
struct TcMap {
    int mrows, ncols, rat, rskip, cat, cskip, beta0_lo, beta0_n, beta0_all;
    int only_lo, only_n, skip_lo, skip_n, kchunks;
    const unsigned *amax;   // [2]: the float bits of the largest entries packed into A and B
};

// tile t of the product -> (tile row, tile column)
// Tiles run column by column (t -> tile row t % ntm of tile column t / ntm): a
// wave of CTAs shares one B tile (the larger, 2x expanded operand) and sweeps
// the A panel, which stays in L2 beside the C column streaming through.
__device__ __forceinline__ void tc_tile(const TcMap &mp, int ntx, int t, int &ty, int &tx) {
    const int ntm = (mp.mrows + TC_TM - 1) / TC_TM;
    ty = t % ntm;
    const int i = t / ntm;
    tx = mp.only_n > 0 ? mp.only_lo + i : (mp.skip_n > 0 && i >= mp.skip_lo ? i + mp.skip_n : i);
}

// C <- beta C + Ap * Bp^T over the tiles of the map.  tmA, tmB: the packed
// operands (box 32 floats x 128 / 256 rows);
// tmC: the block [n rows][2 ld floats] (box 32 x 128, loads); tmCs: the same
// with a 32 x 32 box (stores of one epilogue warp).  All four use SWIZZLE_128B.
// The maps span whole padded rows (a multiple of 16 bytes), so a box that
// reaches past column n stays in bounds: there, and on pivot rows or columns
// that a ragged tile covers, the packed operands are zero and the store writes
// back the value it loaded.
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_update(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmCs, const TcMap mp,
                int *err) {
    extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;                                              // [stage] 16 KB
    uint8_t *sB = sA + TC_STAGES * TC_A_BYTES;                       // [stage] 32 KB
    uint8_t *sC = sB + TC_STAGES * TC_B_BYTES;                       // [slot] 16 KB
    uint64_t *bars = reinterpret_cast<uint64_t *>(sC + TC_CSLOTS * TC_C_BYTES);
    uint64_t *full = bars, *empty = full + TC_STAGES;
    uint64_t *cfull = empty + TC_STAGES, *cempty = cfull + TC_CSLOTS;
    uint64_t *accfull = cempty + TC_CSLOTS, *accempty = accfull + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accempty + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntm = (mp.mrows + TC_TM - 1) / TC_TM, nt = (mp.ncols + TC_TN - 1) / TC_TN;
    const int ntx = mp.only_n > 0 ? mp.only_n : (mp.skip_n > 0 ? nt - mp.skip_n : nt);   // tile columns covered
    const int ntiles = ntm * ntx;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) { mbar_init(full + s, 1); mbar_init(empty + s, 1); }
        for (int s = 0; s < TC_CSLOTS; ++s) { mbar_init(cfull + s, 1); mbar_init(cempty + s, 4); }
        for (int b = 0; b < 2; ++b) { mbar_init(accfull + b, 1); mbar_init(accempty + b, 4); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmC)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmCs)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---- A/B producer -------------------------------------------------------
        int it = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            int ty, tx;
            tc_tile(mp, ntx, t, ty, tx);
            for (int kc = 0; kc < mp.kchunks; ++kc, ++it) {
                const int s = it % TC_STAGES;
                if (it >= TC_STAGES && !mbar_wait(empty + s, (uint32_t)((it / TC_STAGES - 1) & 1))) { ok = false; break; }
                mbar_expect_tx(full + s, TC_A_BYTES + TC_B_BYTES);
                tma_load_2d(sA + s * TC_A_BYTES, &tmA, kc * TC_KCHUNK, ty * TC_TM, full + s);
                tma_load_2d(sB + s * TC_B_BYTES, &tmB, kc * TC_KCHUNK, 2 * tx * TC_TN, full + s);
            }
        }
        if (!ok) atomicOr(err, 2);
        // the loads issued last into each stage have landed before the CTA leaves
        for (int s = 0; s < TC_STAGES; ++s) {
            const int uses = it / TC_STAGES + (s < it % TC_STAGES ? 1 : 0);
            if (uses > 0) mbar_wait(full + s, (uint32_t)((uses - 1) & 1));
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ---------------------------------------------------------
        int it = 0, tl = 0;
        bool ok = true;
        uint64_t *last_bar = nullptr;
        uint32_t last_par = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
            const int b = tl & 1;
            if (tl >= 2 && !mbar_wait(accempty + b, (uint32_t)((tl / 2 - 1) & 1))) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dcol = tmem + (uint32_t)(b * 256);
            for (int kc = 0; kc < mp.kchunks; ++kc, ++it) {
                const int s = it % TC_STAGES;
                if (!mbar_wait(full + s, (uint32_t)((it / TC_STAGES) & 1))) { ok = false; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(sA + s * TC_A_BYTES), b0 = smem_u32(sB + s * TC_B_BYTES);
#pragma unroll
                for (int q = 0; q < TC_KCHUNK / 16; ++q) {   // K = 16 per MMA, 32 bytes along the row
                    const uint64_t da = make_desc(a0 + q * 32), db = make_desc(b0 + q * 32);
                    const uint32_t acc = (kc > 0 || q > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                        ::"r"(dcol), "l"(da), "l"(db), "r"(TC_IDESC), "r"(acc));
                }
                mma_commit(empty + s);   // frees the stage once these MMAs have read it
                last_bar = empty + s;
                last_par = (uint32_t)((it / TC_STAGES) & 1);
            }
            if (!ok) break;
            mma_commit(accfull + b);     // accumulator b complete
            last_bar = accfull + b;
            last_par = (uint32_t)((tl / 2) & 1);
        }
        if (!ok) atomicOr(err, 2);
        // the MMAs issued last have finished before the tensor memory is released
        if (last_bar) mbar_wait(last_bar, last_par);
    } else if (warp == 2 && lane == 0) {
        // ---- C producer ---------------------------------------------------------
        int ci = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            int ty, tx;
            tc_tile(mp, ntx, t, ty, tx);
            const int r0 = ty * TC_TM, c0 = tx * TC_TN;
            const int gr0 = r0 < mp.rat ? r0 : r0 + mp.rskip, gc0 = c0 < mp.cat ? c0 : c0 + mp.cskip;
            for (int cc = 0; cc < TC_CCHUNK; ++cc, ++ci) {
                const int s = ci % TC_CSLOTS;
                if (ci >= TC_CSLOTS && !mbar_wait(cempty + s, (uint32_t)((ci / TC_CSLOTS - 1) & 1))) { ok = false; break; }
                mbar_expect_tx(cfull + s, TC_C_BYTES);
                tma_load_2d(sC + s * TC_C_BYTES, &tmC, 2 * gc0 + cc * 32, gr0, cfull + s);
            }
        }
        if (!ok) atomicOr(err, 2);
        for (int s = 0; s < TC_CSLOTS; ++s) {
            const int uses = ci / TC_CSLOTS + (s < ci % TC_CSLOTS ? 1 : 0);
            if (uses > 0) mbar_wait(cfull + s, (uint32_t)((uses - 1) & 1));
        }
    } else if (warp >= 4) {
        // ---- epilogue: TMEM lane = row; warp q owns rows 32q..32q+31 of the tile --
        const int q4 = warp - 4;
        const int row = q4 * 32 + lane;
        const float unscale = tc_pow2(-tc_shift(mp.amax[0])) * tc_pow2(-tc_shift(mp.amax[1]));   // exact: powers of two
        int ci = 0, tl = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
            int ty, tx;
            tc_tile(mp, ntx, t, ty, tx);
            const int r0 = ty * TC_TM, c0 = tx * TC_TN;
            const int gr0 = r0 < mp.rat ? r0 : r0 + mp.rskip, gc0 = c0 < mp.cat ? c0 : c0 + mp.cskip;
            const bool keep = !(mp.beta0_all || (ty >= mp.beta0_lo && ty < mp.beta0_lo + mp.beta0_n));   // beta = 1
            const int b = tl & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(accfull + b, (uint32_t)((tl / 2) & 1)))) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int cc = 0; cc < TC_CCHUNK; ++cc, ++ci) {
                const int s = ci % TC_CSLOTS;
                if (!__all_sync(0xffffffffu, mbar_wait(cfull + s, (uint32_t)((ci / TC_CSLOTS) & 1)))) { ok = false; break; }
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * 256 + cc * 32);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                      "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                      "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                // the chunk's row `row`: 8 swizzled 16-byte pieces (piece q at q ^ (row & 7))
                uint8_t *rp = sC + s * TC_C_BYTES + row * 128;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float4 *p = reinterpret_cast<float4 *>(rp + ((q ^ (row & 7)) << 4));
                    float4 c = keep ? *p : make_float4(0.f, 0.f, 0.f, 0.f);
                    c.x = fmaf(unscale, __uint_as_float(v[4 * q]), c.x);
                    c.y = fmaf(unscale, __uint_as_float(v[4 * q + 1]), c.y);
                    c.z = fmaf(unscale, __uint_as_float(v[4 * q + 2]), c.z);
                    c.w = fmaf(unscale, __uint_as_float(v[4 * q + 3]), c.w);
                    *p = c;
                }
                // make the generic-proxy writes visible to the bulk copy, then store the warp's rows
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    tma_store_2d(&tmCs, sC + s * TC_C_BYTES + q4 * 32 * 128, 2 * gc0 + cc * 32, gr0 + q4 * 32);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    // the store of the previous chunk has finished reading its slot
                    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                    if (ci > 0) mbar_arrive(cempty + (ci - 1) % TC_CSLOTS);
                }
                __syncwarp();
            }
            if (!ok) break;
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(accempty + b);
        }
        if (!ok && lane == 0) atomicOr(err, 2);
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
    }
}

}  // namespace vie
