// Complex FP32 GEMM update C -= A B on the 5th-generation tensor cores
// (tcgen05, kind::tf32, accumulator in tensor memory), for the Gauss-Jordan
// inversion of the domain blocks of Eq. (6).
//
// A complex product is one real product of the real views:
//   C_rv (M x 2N) = A_rv (M x 2K) * Bt (2K x 2N),  Bt[2k][2n] = Re B, Bt[2k][2n+1] = Im B,
//   Bt[2k+1][2n] = -Im B, Bt[2k+1][2n+1] = Re B,
// where the real view of a row-major complex matrix interleaves (re, im).
//
// One CTA (256 threads) computes a 128 x 128 complex tile (128 x 256 real,
// 256 TMEM columns; two CTAs fit one SM) for any K <= TC_KMAX complex.  K is
// streamed in chunks of 16 complex through two shared-memory stages in the
// K-major 128-byte-swizzle layout (8-row x 128-byte atoms, 16-byte chunks
// XOR-ed with the row index); the MMAs (M=128, N=256, K=8) of a chunk are
// issued by one thread and committed to the stage's mbarrier, which the
// staging of the chunk two steps later waits on.  The accumulator is read back
// with tcgen05.ld and subtracted from C.  Every wait has an iteration limit;
// on timeout the CTA records an error flag, skips its update and still frees
// its tensor memory.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace vie {

constexpr int TC_TM = 128;            // complex rows per tile
constexpr int TC_TN = 128;            // complex columns per tile (256 real)
constexpr int TC_KMAX = 128;          // complex K per launch (pivot block width)
constexpr int TC_CHUNK = 32;          // real K elements per stage (one 128-byte swizzle row)
constexpr int TC_A_CHUNK_BYTES = TC_TM * 128;          // 16 KB
constexpr int TC_B_CHUNK_BYTES = 2 * TC_TN * 128;      // 32 KB
constexpr int TC_STAGES = 2;
constexpr int TC_SMEM = TC_STAGES * (TC_A_CHUNK_BYTES + TC_B_CHUNK_BYTES) + 1024 + 64;   // ~97 KB: 2 CTAs/SM
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr long long TC_WAIT_LIMIT = 20000000;  // ~ tens of ms of polling
constexpr int TC_THREADS = 256;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of real element (row r, k in [0,32)) inside one swizzled chunk
__device__ __forceinline__ uint32_t sw128(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) + ((k & 3) << 2));
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

// instruction descriptor: D f32, A/B tf32, K-major, N = 256, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// One Gauss-Jordan trailing update on the tile (blockIdx.y, blockIdx.x):
// C[r][c] -= sum_k C[r][k0+k] C[k0+k][c] for k < K, over rows and columns
// outside the pivot block [k0, k0+w): tile row i maps to r = i < k0 ? i : i + w
// (columns likewise), m = n - w rows and columns are updated.  The pivot rows
// and columns are only read, so tiles never race.
// bounded wait on an mbarrier phase; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity) {
    for (long long it = 0; it < TC_WAIT_LIMIT; ++it) {
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

__global__ void __launch_bounds__(TC_THREADS) k_tc_update(float *__restrict__ C, size_t ld, int m, int k0, int w,
                                                          int K, int *err) {
    extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;                                         // [stage] 16 KB
    uint8_t *sB = base + TC_STAGES * TC_A_CHUNK_BYTES;          // [stage] 32 KB
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sB + TC_STAGES * TC_B_CHUNK_BYTES);   // [stage]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + TC_STAGES);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ti = blockIdx.y * TC_TM, tj = blockIdx.x * TC_TN;
    const int nch = (2 * K + TC_CHUNK - 1) / TC_CHUNK;   // stages of 16 complex k

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + s)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    // per-thread registers of one chunk: A items (row, k pair) and B items (column, k pair)
    constexpr int NA = TC_TM * 8 / TC_THREADS, NB = TC_TN * 8 / TC_THREADS;   // 4 and 4
    float4 ra[NA];
    float4 rb[NB];   // (Re B[k], Im B[k], Re B[k+1], Im B[k+1]) of one column
    auto load_chunk = [&](int c) {
        const int kc0 = c * (TC_CHUNK / 2);
        const int kcn = min(TC_CHUNK / 2, K - kc0);
#pragma unroll
        for (int u = 0; u < NA; ++u) {
            const int e = tid + u * TC_THREADS;
            const int i = e >> 3, f = e & 7;
            const int ii = ti + i;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ii < m && 2 * f < kcn) {
                const int r = ii < k0 ? ii : ii + w;
                const float *src = C + 2 * ((size_t)r * ld + k0 + kc0 + 2 * f);
                if (2 * f + 1 < kcn) v = __ldcg(reinterpret_cast<const float4 *>(src));
                else v = make_float4(__ldcg(src), __ldcg(src + 1), 0.f, 0.f);
            }
            ra[u] = v;
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int e = tid + u * TC_THREADS;
            const int j = e % TC_TN, kp = e / TC_TN;
            const int jj = tj + j;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (jj < m && 2 * kp < kcn) {
                const int cc = jj < k0 ? jj : jj + w;
                const float2 u0 = __ldcg(reinterpret_cast<const float2 *>(C + 2 * ((size_t)(k0 + kc0 + 2 * kp) * ld + cc)));
                v.x = u0.x;
                v.y = u0.y;
                if (2 * kp + 1 < kcn) {
                    const float2 u1 =
                        __ldcg(reinterpret_cast<const float2 *>(C + 2 * ((size_t)(k0 + kc0 + 2 * kp + 1) * ld + cc)));
                    v.z = u1.x;
                    v.w = u1.y;
                }
            }
            rb[u] = v;
        }
    };
    auto store_chunk = [&](uint8_t *a_st, uint8_t *b_st) {
#pragma unroll
        for (int u = 0; u < NA; ++u) {
            const int e = tid + u * TC_THREADS;
            const int i = e >> 3, f = e & 7;
            const float4 v = ra[u];
            *reinterpret_cast<float4 *>(a_st + sw128(i, 4 * f)) =
                make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
            const int e = tid + u * TC_THREADS;
            const int j = e % TC_TN, kp = e / TC_TN;
            const float4 v = rb[u];
            // real column 2j (Re C): [Re B, -Im B]; column 2j+1 (Im C): [Im B, Re B]
            *reinterpret_cast<float4 *>(b_st + sw128(2 * j, 4 * kp)) =
                make_float4(to_tf32(v.x), to_tf32(-v.y), to_tf32(v.z), to_tf32(-v.w));
            *reinterpret_cast<float4 *>(b_st + sw128(2 * j + 1, 4 * kp)) =
                make_float4(to_tf32(v.y), to_tf32(v.x), to_tf32(v.w), to_tf32(v.z));
        }
    };

    load_chunk(0);
    for (int c = 0; c < nch; ++c) {
        const int st = c % TC_STAGES;
        uint8_t *a_st = sA + st * TC_A_CHUNK_BYTES;
        uint8_t *b_st = sB + st * TC_B_CHUNK_BYTES;
        if (c >= TC_STAGES) {   // the MMAs of chunk c-2 read this stage: wait for them
            bool done = mbar_wait(mbar + st, (uint32_t)(((c - TC_STAGES) / TC_STAGES) & 1));
            ok = __syncthreads_and(done) && ok;
            if (!ok) break;
        }
        store_chunk(a_st, b_st);
        if (c + 1 < nch) load_chunk(c + 1);   // next chunk's loads overlap this chunk's MMAs
        // make the generic-proxy shared stores visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const int kcn = min(TC_CHUNK / 2, K - c * (TC_CHUNK / 2));
            const int steps = (2 * kcn + 7) / 8;
            for (int s2 = 0; s2 < steps; ++s2) {
                const uint64_t da = make_desc(smem_u32(a_st) + s2 * 32), db = make_desc(smem_u32(b_st) + s2 * 32);
                const uint32_t acc = (c > 0 || s2 > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                    ::"r"(tmem), "l"(da), "l"(db), "r"(TC_IDESC), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         ::"r"(smem_u32(mbar + st)) : "memory");
        }
    }
    // wait for the last chunk (in-order completion covers the earlier ones)
    if (ok) {
        const int last = nch - 1;
        bool done = mbar_wait(mbar + (last % TC_STAGES), (uint32_t)((last / TC_STAGES) & 1));
        ok = __syncthreads_and(done);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        // record the failure and give the MMAs in flight a second bounded wait
        // before the tensor memory is released; the update is skipped
        if (tid == 0) atomicExch(err, 2);
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_wait(mbar + s, 0);
            mbar_wait(mbar + s, 1);
        }
    } else {
        // ---- epilogue: TMEM (row = lane) -> registers -> C -= acc ------------------
        const int i = (warp & 3) * 32 + lane;
        const int ii = ti + i;
        const int r = ii < k0 ? ii : ii + w;
        const int cbase = (warp >> 2) * 128;   // warps 4..7 take real columns 128..255
        for (int c0 = cbase; c0 < cbase + 128; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (ii >= m) continue;
            // 16 complex columns jj = tj + c0/2 + q, as 8 pairs
            float4 old[8];
            bool vec[8];
#pragma unroll
            for (int p2 = 0; p2 < 8; ++p2) {
                const int jj = tj + c0 / 2 + 2 * p2;
                const int cc = jj < k0 ? jj : jj + w;
                vec[p2] = (jj + 1 < m) && !(jj < k0 && jj + 1 >= k0) && (cc & 1) == 0;
                if (vec[p2]) old[p2] = __ldcs(reinterpret_cast<const float4 *>(C + 2 * ((size_t)r * ld + cc)));
            }
#pragma unroll
            for (int p2 = 0; p2 < 8; ++p2) {
                const int jj = tj + c0 / 2 + 2 * p2;
                const float a0 = __uint_as_float(v[4 * p2]), a1 = __uint_as_float(v[4 * p2 + 1]);
                const float a2 = __uint_as_float(v[4 * p2 + 2]), a3 = __uint_as_float(v[4 * p2 + 3]);
                if (vec[p2]) {
                    const int cc = jj < k0 ? jj : jj + w;
                    float4 o = old[p2];
                    o.x -= a0; o.y -= a1; o.z -= a2; o.w -= a3;
                    __stcs(reinterpret_cast<float4 *>(C + 2 * ((size_t)r * ld + cc)), o);   // streaming: keep the panels in L2
                } else {
                    for (int h = 0; h < 2; ++h) {
                        const int j2 = jj + h;
                        if (j2 >= m) break;
                        const int c2 = j2 < k0 ? j2 : j2 + w;
                        float *pp = C + 2 * ((size_t)r * ld + c2);
                        pp[0] -= h ? a2 : a0;
                        pp[1] -= h ? a3 : a1;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
    }
}

}  // namespace vie
