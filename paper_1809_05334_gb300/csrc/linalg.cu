// Dense complex linear algebra of the solve: the HBM-bound matvec Y = Z X for
// two right-hand sides, the in-place blocked Gauss-Jordan inversion of the
// domain blocks A_dd of Eq. (6) (no pivoting), and the vector kernels of GMRES.
//
// Layouts: complex interleaved (re, im).  A matrix is `rows` rows of `ld`
// complex entries (ld a multiple of 4, zero padded).  Vectors with two
// right-hand sides are [n][2] complex.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "linalg.h"
#include "tc_gemm.cuh"

namespace vie {

template <typename T> struct V2;
template <> struct V2<float> { using t = float4; };
template <> struct V2<double> { using t = double2; };
template <> struct V2<__half> { using t = uint4; };   // four complex FP16 entries
template <> struct V2<__nv_bfloat16> { using t = uint4; };   // four complex BF16 entries

// one complex 16-bit entry (two halves of a 32-bit word) widened to FP32
template <typename T> __device__ __forceinline__ float2 widen2(uint32_t w);
template <> __device__ __forceinline__ float2 widen2<__half>(uint32_t w) {
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}
template <> __device__ __forceinline__ float2 widen2<__nv_bfloat16>(uint32_t w) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
}

// ---------------------------------------------------------------------------
// matvec: y[r] = alpha sum_c A[r][c] x[c] (+ y[r] if ACCUM) for rows [0, rows),
// two right-hand sides ([n][2] complex vectors).
// The grid is one wave (every resident CTA slot of the GPU); CTA b owns the
// contiguous rows [rows b / G, rows (b+1) / G), so all CTAs stream the same
// number of bytes.  Its warps split the columns of each group of MV_ROWS rows
// (equal segments, 16-byte loads of A streamed with evict-first), reduce by
// shuffles, and combine the warps' partial sums through shared memory (double
// buffered: one barrier per row group).  x is read through L1/L2 (it is a few
// hundred KB and every row group reuses it).  16-bit entries carry twice the
// products per byte, so their loop keeps the next column step's loads in
// flight while it multiplies the current ones (80 registers, three CTAs per
// SM); FP32 and FP64 entries rely on the unrolled loop alone.
// ---------------------------------------------------------------------------
constexpr int MV_ROWS = 4;
constexpr int MV_WARPS = 8;

template <typename TX, typename TA> __device__ __forceinline__ void load_x(const TX *x, int c, TA out[4]);
template <> __device__ __forceinline__ void load_x<float, float>(const float *x, int c, float out[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(x + 4 * (size_t)c));
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <> __device__ __forceinline__ void load_x<double, double>(const double *x, int c, double out[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(x + 4 * (size_t)c));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(x + 4 * (size_t)c + 2));
    out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}

template <typename TZ, typename TX, typename TA, bool ACCUM>
__global__ void __launch_bounds__(MV_WARPS * 32)
k_matvec(const TZ *__restrict__ A, size_t ld, int rows, int cols, const TX *__restrict__ x,
         TA *__restrict__ y, TA alpha) {
    __shared__ TA part[2][MV_WARPS][MV_ROWS * 4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rb = (int)((long long)rows * blockIdx.x / gridDim.x);
    const int re = (int)((long long)rows * (blockIdx.x + 1) / gridDim.x);
    constexpr int VEC = sizeof(TZ) == 4 ? 2 : (sizeof(TZ) == 8 ? 1 : 4);   // complex entries per 16-byte load
    // 16-bit entries: the column-interleaved layout (ld16 columns per row, load
    // v holds columns 128 (v / 32) + v % 32 + 32 u); warp segments start on a
    // chunk, so a warp's x loads of one step are contiguous
    const int nvec = VEC == 4 ? (cols + 127) / 128 * 32 : (cols + VEC - 1) / VEC;
    int v0 = (int)((long long)nvec * warp / MV_WARPS), v1 = (int)((long long)nvec * (warp + 1) / MV_WARPS);
    if (VEC == 4) {
        v0 &= ~31;
        v1 = warp + 1 == MV_WARPS ? nvec : (v1 & ~31);
    }
    int buf = 0;
    for (int r0 = rb; r0 < re; r0 += MV_ROWS, buf ^= 1) {
        TA acc[MV_ROWS][4];
#pragma unroll
        for (int i = 0; i < MV_ROWS; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][k] = TA(0);
        auto zload = [&](int v, typename V2<TZ>::t *z) {
            const int c = v * VEC;
#pragma unroll
            for (int i = 0; i < MV_ROWS; ++i) {
                if (r0 + i < re)
                    z[i] = __ldcs(reinterpret_cast<const typename V2<TZ>::t *>(A + 2 * ((size_t)(r0 + i) * ld + c)));
                else
                    z[i] = {};
            }
        };
        auto zuse = [&](int v, const typename V2<TZ>::t *z) {
            const int c = v * VEC;
#pragma unroll
            for (int u = 0; u < VEC; ++u) {
                TA xv[4] = {TA(0), TA(0), TA(0), TA(0)};
                const int cu = VEC == 4 ? (v >> 5) * 128 + (v & 31) + 32 * u : c + u;   // the entry's column
                if (cu < cols) load_x<TX, TA>(x, cu, xv);
#pragma unroll
                for (int i = 0; i < MV_ROWS; ++i) {
                    TA zr, zi;
                    if constexpr (VEC == 4) {
                        const uint32_t *wv = reinterpret_cast<const uint32_t *>(&z[i]);
                        const float2 f = widen2<TZ>(wv[u]);
                        zr = TA(f.x);
                        zi = TA(f.y);
                    } else if constexpr (VEC == 2) {
                        const float4 f = *reinterpret_cast<const float4 *>(&z[i]);
                        zr = TA(u == 0 ? f.x : f.z);
                        zi = TA(u == 0 ? f.y : f.w);
                    } else {
                        const double2 d = *reinterpret_cast<const double2 *>(&z[i]);
                        zr = TA(d.x);
                        zi = TA(d.y);
                    }
                    acc[i][0] = fma(zr, xv[0], fma(-zi, xv[1], acc[i][0]));
                    acc[i][1] = fma(zr, xv[1], fma(zi, xv[0], acc[i][1]));
                    acc[i][2] = fma(zr, xv[2], fma(-zi, xv[3], acc[i][2]));
                    acc[i][3] = fma(zr, xv[3], fma(zi, xv[2], acc[i][3]));
                }
            }
        };
        if constexpr (VEC == 4) {   // 16-bit entries: the next column step's loads in flight during this one's products
            typename V2<TZ>::t zc[MV_ROWS], zn[MV_ROWS];
            int v = v0 + lane;
            if (v < v1) zload(v, zc);
#pragma unroll 2
            for (; v < v1; v += 32) {
                if (v + 32 < v1) zload(v + 32, zn);
                else {
#pragma unroll
                    for (int i = 0; i < MV_ROWS; ++i) zn[i] = {};
                }
                zuse(v, zc);
#pragma unroll
                for (int i = 0; i < MV_ROWS; ++i) zc[i] = zn[i];
            }
        } else {
#pragma unroll 8
            for (int v = v0 + lane; v < v1; v += 32) {
                typename V2<TZ>::t z[MV_ROWS];
                zload(v, z);
                zuse(v, z);
            }
        }
#pragma unroll
        for (int i = 0; i < MV_ROWS; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[i][k] += __shfl_down_sync(0xffffffffu, acc[i][k], o);
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < MV_ROWS; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) part[buf][warp][4 * i + k] = acc[i][k];
        }
        __syncthreads();
        if (threadIdx.x < MV_ROWS * 4) {
            const int i = threadIdx.x / 4, k = threadIdx.x % 4;
            const int r = r0 + i;
            if (r < re) {
                TA s = TA(0);
#pragma unroll
                for (int w2 = 0; w2 < MV_WARPS; ++w2) s += part[buf][w2][threadIdx.x];
                if (ACCUM) y[(size_t)r * 4 + k] += alpha * s;
                else y[(size_t)r * 4 + k] = alpha * s;
            }
        }
    }
}

template <typename TZ, typename TX, typename TA>
cudaError_t matvec(const TZ *A, size_t ld, int rows, int cols, const TX *x, TA *y, TA alpha, bool accumulate,
                   cudaStream_t st, int grid_mult) {
    if (rows <= 0) return cudaSuccess;
    static int slots = 0;   // resident CTAs of the GPU (per instantiation; one device per process)
    if (slots == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_matvec<TZ, TX, TA, false>, MV_WARPS * 32, 0);
        if (e != cudaSuccess) return e;
        slots = std::max(1, sms * per);
    }
    // grid_mult > 1: that many row ranges per resident CTA (finer ranges, a shorter tail)
    const int grid = std::max(1, std::min(slots * std::max(1, grid_mult), (rows + MV_ROWS - 1) / MV_ROWS));
    if (accumulate)
        k_matvec<TZ, TX, TA, true><<<grid, MV_WARPS * 32, 0, st>>>(A, ld, rows, cols, x, y, alpha);
    else
        k_matvec<TZ, TX, TA, false><<<grid, MV_WARPS * 32, 0, st>>>(A, ld, rows, cols, x, y, alpha);
    ++g_launches;
    return cudaGetLastError();
}

template cudaError_t matvec<float, float, float>(const float *, size_t, int, int, const float *, float *, float, bool, cudaStream_t, int);
template cudaError_t matvec<__half, float, float>(const __half *, size_t, int, int, const float *, float *, float, bool, cudaStream_t, int);
template cudaError_t matvec<__half, double, double>(const __half *, size_t, int, int, const double *, double *, double, bool,
                                                    cudaStream_t, int);
template cudaError_t matvec<__nv_bfloat16, float, float>(const __nv_bfloat16 *, size_t, int, int, const float *, float *,
                                                         float, bool, cudaStream_t, int);

// largest |Re|, |Im| of a block, as the bit pattern of a non-negative float
// (for those the integer order is the float order, so atomicMax applies)
__global__ void k_absmax(const float *__restrict__ A, size_t count, unsigned *out) {
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(A[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// B = scale A in 16 bits (round to nearest), column-interleaved: one thread per
// complex entry of B (rows x ld16(cols)); position p of a row holds column
// chunk + (p % 4) * 32 + (p % 128) / 4, zero past cols
template <typename T>
__global__ void k_to16_il(const float *__restrict__ A, size_t lda, int rows, int cols, float scale, T *__restrict__ B) {
    const size_t ldb = ((size_t)cols + 127) / 128 * 128;
    const size_t total = (size_t)rows * ldb;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / ldb, p = i - r * ldb;
        const size_t pp = p & 127;
        const size_t c = (p - pp) + (pp & 3) * 32 + (pp >> 2);
        float2 v = make_float2(0.f, 0.f);
        if (c < (size_t)cols) v = *reinterpret_cast<const float2 *>(A + 2 * (r * lda + c));
        if constexpr (sizeof(T) == 2 && std::is_same<T, __half>::value) {
            B[2 * i] = __float2half_rn(v.x * scale);
            B[2 * i + 1] = __float2half_rn(v.y * scale);
        } else {
            B[2 * i] = __float2bfloat16_rn(v.x);
            B[2 * i + 1] = __float2bfloat16_rn(v.y);
        }
    }
}

cudaError_t to_bf16_il(const float *A, size_t lda, int rows, int cols, __nv_bfloat16 *B, cudaStream_t st) {
    k_to16_il<__nv_bfloat16><<<1216, 256, 0, st>>>(A, lda, rows, cols, 1.f, B); ++g_launches;
    return cudaGetLastError();
}

cudaError_t to_half_il(const float *A, size_t lda, int rows, int cols, float scale, __half *B, cudaStream_t st) {
    k_to16_il<__half><<<1216, 256, 0, st>>>(A, lda, rows, cols, scale, B); ++g_launches;
    return cudaGetLastError();
}

cudaError_t absmax(const float *A, size_t count, unsigned *out, cudaStream_t st) {
    k_absmax<<<1216, 256, 0, st>>>(A, count, out); ++g_launches;
    return cudaGetLastError();
}

template cudaError_t matvec<float, double, double>(const float *, size_t, int, int, const double *, double *, double, bool, cudaStream_t, int);

// ---------------------------------------------------------------------------
// Residual product of the FP64 refinement, y <- y + alpha Z x, Z in FP32 and
// x, y in FP64, without FP64 arithmetic in the inner loop (the FP64 pipe is a
// small fraction of the FP32 one): x is split once into x = xh + xl (two FP32
// parts, 48 significant bits), every product Z xh is formed exactly as p + e
// (p = Z xh rounded, e = fma(Z, xh, -p)), the p are summed with TwoSum into a
// running (S, C) pair per output value, and e and the small Z xl terms go into
// C.  The result carries the error of a double-length sum (~2^-44 of the sum
// of |terms|), far below the FP32 rounding of Z itself.  Same row and column
// split as k_matvec.
// ---------------------------------------------------------------------------
__global__ void k_split_x(const double *__restrict__ x, float *__restrict__ xs, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * n) return;
    const double v = x[i];
    const float h = (float)v;
    const float l = (float)(v - (double)h);
    const int r = i / 4, k = i % 4;
    xs[8 * (size_t)r + k] = h;
    xs[8 * (size_t)r + 4 + k] = l;
}

struct DS {   // unevaluated sum S + C
    float s, c;
};
__device__ __forceinline__ void ds_add(DS &a, float p) {   // a += p (TwoSum on the leading part)
    const float t = __fadd_rn(a.s, p);
    const float bp = __fsub_rn(t, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    a.s = t;
    a.c = __fadd_rn(a.c, err);
}
// a += z * xh + z * xl, the first product exact (p + e)
__device__ __forceinline__ void ds_fma(DS &a, float z, float xh, float xl) {
    const float p = __fmul_rn(z, xh);
    const float e = __fmaf_rn(z, xh, -p);
    ds_add(a, p);
    a.c = __fmaf_rn(z, xl, __fadd_rn(a.c, e));
}
__device__ __forceinline__ DS ds_sum(DS a, DS b) {
    DS r = a;
    ds_add(r, b.s);
    r.c = __fadd_rn(r.c, b.c);
    return r;
}

template <bool ACCUM>
__global__ void __launch_bounds__(MV_WARPS * 32)
k_matvec_ds(const float *__restrict__ A, size_t ld, int rows, int cols, const float *__restrict__ xs,
            double *__restrict__ y, double alpha) {
    __shared__ double part[2][MV_WARPS][MV_ROWS * 4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rb = (int)((long long)rows * blockIdx.x / gridDim.x);
    const int re = (int)((long long)rows * (blockIdx.x + 1) / gridDim.x);
    const int nvec = (cols + 1) / 2;   // two complex FP32 entries per 16-byte load
    const int v0 = (int)((long long)nvec * warp / MV_WARPS), v1 = (int)((long long)nvec * (warp + 1) / MV_WARPS);
    int buf = 0;
    for (int r0 = rb; r0 < re; r0 += MV_ROWS, buf ^= 1) {
        DS acc[MV_ROWS][4];
#pragma unroll
        for (int i = 0; i < MV_ROWS; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][k] = {0.f, 0.f};
        for (int v = v0 + lane; v < v1; v += 32) {
            const int c = 2 * v;
            float4 z[MV_ROWS];
#pragma unroll
            for (int i = 0; i < MV_ROWS; ++i) {
                if (r0 + i < re) z[i] = __ldcs(reinterpret_cast<const float4 *>(A + 2 * ((size_t)(r0 + i) * ld + c)));
                else z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
                if (c + u < cols) {
                    h = __ldg(reinterpret_cast<const float4 *>(xs + 8 * (size_t)(c + u)));
                    l = __ldg(reinterpret_cast<const float4 *>(xs + 8 * (size_t)(c + u) + 4));
                }
#pragma unroll
                for (int i = 0; i < MV_ROWS; ++i) {
                    const float zr = u == 0 ? z[i].x : z[i].z, zi = u == 0 ? z[i].y : z[i].w;
                    // (zr + j zi)(xr + j xi) for the two right-hand sides
                    ds_fma(acc[i][0], zr, h.x, l.x);
                    ds_fma(acc[i][0], -zi, h.y, l.y);
                    ds_fma(acc[i][1], zr, h.y, l.y);
                    ds_fma(acc[i][1], zi, h.x, l.x);
                    ds_fma(acc[i][2], zr, h.z, l.z);
                    ds_fma(acc[i][2], -zi, h.w, l.w);
                    ds_fma(acc[i][3], zr, h.w, l.w);
                    ds_fma(acc[i][3], zi, h.z, l.z);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < MV_ROWS; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    DS b;
                    b.s = __shfl_down_sync(0xffffffffu, acc[i][k].s, o);
                    b.c = __shfl_down_sync(0xffffffffu, acc[i][k].c, o);
                    acc[i][k] = ds_sum(acc[i][k], b);
                }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < MV_ROWS; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) part[buf][warp][4 * i + k] = (double)acc[i][k].s + (double)acc[i][k].c;
        }
        __syncthreads();
        if (threadIdx.x < MV_ROWS * 4) {
            const int i = threadIdx.x / 4, k = threadIdx.x % 4;
            const int r = r0 + i;
            if (r < re) {
                double s = 0.0;
#pragma unroll
                for (int w2 = 0; w2 < MV_WARPS; ++w2) s += part[buf][w2][threadIdx.x];
                if (ACCUM) y[(size_t)r * 4 + k] += alpha * s;
                else y[(size_t)r * 4 + k] = alpha * s;
            }
        }
    }
}

cudaError_t matvec_ds(const float *A, size_t ld, int rows, int cols, const double *x, float *xs, double *y,
                      double alpha, bool accumulate, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    static int slots = 0;   // resident CTAs of the GPU (one device per process)
    if (slots == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_matvec_ds<false>, MV_WARPS * 32, 0);
        if (e != cudaSuccess) return e;
        slots = std::max(1, sms * per);
    }
    k_split_x<<<(4 * cols + 255) / 256, 256, 0, st>>>(x, xs, cols); ++g_launches;
    const int grid = std::max(1, std::min(slots, (rows + MV_ROWS - 1) / MV_ROWS));
    if (accumulate) k_matvec_ds<true><<<grid, MV_WARPS * 32, 0, st>>>(A, ld, rows, cols, xs, y, alpha);
    else k_matvec_ds<false><<<grid, MV_WARPS * 32, 0, st>>>(A, ld, rows, cols, xs, y, alpha);
    ++g_launches;
    return cudaGetLastError();
}
template cudaError_t matvec<double, double, double>(const double *, size_t, int, int, const double *, double *, double, bool, cudaStream_t, int);

// ---------------------------------------------------------------------------
// Peak of the FP32 / FP64 FMA pipes, for the roofline of the CUDA-core
// kernels: every thread runs FMA_CHAINS independent dependent chains of
// fma(a, x, b) for `iters` steps (2 flops each); the chains hide the pipe
// latency and the result is stored only if it is impossible, so nothing is
// optimised away.
// ---------------------------------------------------------------------------
constexpr int FMA_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T a, T b, int iters, T *sink) {
    T x[FMA_CHAINS];
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int c = 0; c < FMA_CHAINS; ++c) x[c] = fma(a, x[c], b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) s += x[c];
    if (s == T(-1.2345e-29)) sink[blockIdx.x] = s;
}

cudaError_t fma_peak(bool fp64, int iters, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, double *flops) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma_peak<double>, 256, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fma_peak<float>, 256, 0);
    if (e != cudaSuccess) return e;
    const int grid = sms * std::max(per, 1);
    *flops = 2.0 * grid * 256.0 * iters * 16.0 * FMA_CHAINS;
    cudaEventRecord(e0, st);
    if (fp64) k_fma_peak<double><<<grid, 256, 0, st>>>(0.999999, 1e-7, iters, nullptr);
    else k_fma_peak<float><<<grid, 256, 0, st>>>(0.9999f, 1e-4f, iters, nullptr);
    ++g_launches;
    cudaEventRecord(e1, st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Check of the bounded mbarrier wait the tensor-core products use: one thread
// initialises an mbarrier for one arrival, arrives on it or not, and waits on
// its phase 0 with the same bounded wait (at most `polls` polls); a wait that
// runs out sets bit 1 of *status, as a stalled product does.
// ---------------------------------------------------------------------------
__global__ void k_wait_check(int arrive, long long polls, int *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (arrive) mbar_arrive(&bar);
    if (!mbar_wait(&bar, 0, polls)) atomicOr(status, 2);
}

cudaError_t wait_check(bool arrive, long long polls, int *status, cudaStream_t st) {
    k_wait_check<<<1, 32, 0, st>>>(arrive ? 1 : 0, polls, status); ++g_launches;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gauss-Jordan with 512-wide outer pivot blocks and tensor-core products
// (FP32 matrix; FP16 operands scaled by powers of two, FP32 accumulation).
// ---------------------------------------------------------------------------
constexpr int GJ_W = 128;     // pivot block width (the K of the tensor-core update)

// In-place Gauss-Jordan inverse of the w x w (w <= GJ_W) pivot block, held in
// registers, two pivots per step: 512 threads; warp v owns the columns
// c = 32 (v / 4) + lane and the rows g + 4q (g = v % 4, q = 0..31), so the four
// warps that own a column (the pivot columns' owners do the extra work of a
// step) sit on the four schedulers; the block is padded with the identity up
// to an even width.  Step (j, j+1) with the 2 x 2 pivot block P
// and rows R = A[j:j+2, :] is one update of every entry,
//   a_ic <- a_ic - f_i0 m_0c - f_i1 m_1c,
// m_c = P^-1 R[:, c] off the pivot columns and the matching column of P^-1 on
// them; f_i = (a_ij, a_i,j+1) off the pivot rows and the rows of P - I on them;
// the owners of the pivot columns start from the unit vectors.  This gives
// P^-1 R on the pivot rows, P^-1 on the pivot block, -F P^-1 on the pivot
// columns and A - F P^-1 R elsewhere.  The pivot rows and the factors travel
// through double-buffered shared memory; the owners of the next pair publish
// them right after their update, so one barrier per two pivots suffices.
constexpr int GJ_DG = 4;               // row groups of the pivot-block inverse (512 threads)
constexpr int GJ_RQ = GJ_W / GJ_DG;    // rows per thread
__global__ void __launch_bounds__(GJ_W * GJ_DG) k_gj_diag_w(float *A, size_t ld, int k0, int w, int *status) {
    __shared__ float2 rowbuf[2][2][GJ_W];
    __shared__ __align__(16) float2 colbuf[2][GJ_DG][GJ_RQ][2];   // factors (f0, f1) of the pivot pair, row g + 4q
    const int wv = threadIdx.x >> 5;
    const int c = 32 * (wv >> 2) + (threadIdx.x & 31), g = wv & (GJ_DG - 1);
    float2 a[GJ_RQ];
#pragma unroll
    for (int q = 0; q < GJ_RQ; ++q) {
        const int i = g + GJ_DG * q;
        a[q] = make_float2(i == c && (i >= w || c >= w) ? 1.f : 0.f, 0.f);   // identity on the padding
        if (i < w && c < w) a[q] = *reinterpret_cast<const float2 *>(A + 2 * ((size_t)(k0 + i) * ld + k0 + c));
    }
    const int wr = (w + 1) & ~1;
    // pair 0: rows 0, 1 (groups 0, 1, slot 0), columns 0, 1, the diagonal factors minus one
    if (g < 2) rowbuf[0][g][c] = a[0];
    if (c < 2) {
#pragma unroll
        for (int q = 0; q < GJ_RQ; ++q) colbuf[0][g][q][c] = a[q];
        if (g == c) colbuf[0][g][0][c] = make_float2(a[0].x - 1.f, a[0].y);
    }
    for (int j = 0; j < wr; j += 2) {
        const int b = (j >> 1) & 1, nb = b ^ 1, jn = j + 2;
        __syncthreads();
        const float2 p00 = rowbuf[b][0][j], p01 = rowbuf[b][0][j + 1], p10 = rowbuf[b][1][j], p11 = rowbuf[b][1][j + 1];
        const float dr = (p00.x * p11.x - p00.y * p11.y) - (p01.x * p10.x - p01.y * p10.y);
        const float di = (p00.x * p11.y + p00.y * p11.x) - (p01.x * p10.y + p01.y * p10.x);
        const float dd = dr * dr + di * di;
        if (threadIdx.x == 0 && (!(dd > 0.f) || !isfinite(dd))) atomicOr(status, 1);
        const float rd = __frcp_rn(dd);
        const float er = dr * rd, ei = -di * rd;   // 1 / det
        auto cm = [](float ar, float ai, float br, float bi) { return make_float2(ar * br - ai * bi, ar * bi + ai * br); };
        const float2 q00 = cm(p11.x, p11.y, er, ei), q01 = cm(-p01.x, -p01.y, er, ei);
        const float2 q10 = cm(-p10.x, -p10.y, er, ei), q11 = cm(p00.x, p00.y, er, ei);   // P^-1
        float2 m0, m1;
        if (c == j || c == j + 1) {   // a pivot column: m = column of P^-1, entries from the unit vector
            m0 = c == j ? q00 : q01;
            m1 = c == j ? q10 : q11;
#pragma unroll
            for (int q = 0; q < GJ_RQ; ++q) a[q] = make_float2(g + GJ_DG * q == c ? 1.f : 0.f, 0.f);
        } else {
            const float2 r0 = rowbuf[b][0][c], r1 = rowbuf[b][1][c];
            m0 = make_float2(q00.x * r0.x - q00.y * r0.y + q01.x * r1.x - q01.y * r1.y,
                             q00.x * r0.y + q00.y * r0.x + q01.x * r1.y + q01.y * r1.x);
            m1 = make_float2(q10.x * r0.x - q10.y * r0.y + q11.x * r1.x - q11.y * r1.y,
                             q10.x * r0.y + q10.y * r0.x + q11.x * r1.y + q11.y * r1.x);
        }
#pragma unroll
        for (int q = 0; q < GJ_RQ; ++q) {
            const float4 ff = *reinterpret_cast<const float4 *>(&colbuf[b][g][q][0]);
            a[q].x = fmaf(-ff.x, m0.x, fmaf(ff.y, m0.y, fmaf(-ff.z, m1.x, fmaf(ff.w, m1.y, a[q].x))));
            a[q].y = fmaf(-ff.x, m0.y, fmaf(-ff.y, m0.x, fmaf(-ff.z, m1.y, fmaf(-ff.w, m1.x, a[q].y))));
        }
        if (jn < wr) {
            // rows jn, jn + 1: groups jn % 4 and jn % 4 + 1, slot jn / 4
            const int gj = jn & (GJ_DG - 1), qn = jn / GJ_DG;
            if (g == gj || g == gj + 1) {
                float2 r = make_float2(0.f, 0.f);
                switch (qn) {
#define GJ_ROW_CASE(k) case k: r = a[k]; break;
                    GJ_ROW_CASE(0) GJ_ROW_CASE(1) GJ_ROW_CASE(2) GJ_ROW_CASE(3) GJ_ROW_CASE(4) GJ_ROW_CASE(5)
                    GJ_ROW_CASE(6) GJ_ROW_CASE(7) GJ_ROW_CASE(8) GJ_ROW_CASE(9) GJ_ROW_CASE(10) GJ_ROW_CASE(11)
                    GJ_ROW_CASE(12) GJ_ROW_CASE(13) GJ_ROW_CASE(14) GJ_ROW_CASE(15) GJ_ROW_CASE(16) GJ_ROW_CASE(17)
                    GJ_ROW_CASE(18) GJ_ROW_CASE(19) GJ_ROW_CASE(20) GJ_ROW_CASE(21) GJ_ROW_CASE(22) GJ_ROW_CASE(23)
                    GJ_ROW_CASE(24) GJ_ROW_CASE(25) GJ_ROW_CASE(26) GJ_ROW_CASE(27) GJ_ROW_CASE(28) GJ_ROW_CASE(29)
                    GJ_ROW_CASE(30) GJ_ROW_CASE(31)
#undef GJ_ROW_CASE
                    default: break;
                }
                rowbuf[nb][g - gj][c] = r;
            }
            if (c == jn || c == jn + 1) {   // columns jn, jn + 1: the factors, diagonal ones minus one
                const int h = c - jn;
#pragma unroll
                for (int q = 0; q < GJ_RQ; ++q) colbuf[nb][g][q][h] = a[q];
                if (g == gj + h) {
                    const float2 dj = rowbuf[nb][h][c];
                    colbuf[nb][g][qn][h] = make_float2(dj.x - 1.f, dj.y);
                }
            }
        }
    }
    float *Ao;
    asm volatile("mov.b64 %0, %1;" : "=l"(Ao) : "l"(A));
#pragma unroll
    for (int q = 0; q < GJ_RQ; ++q) {
        const int i = g + GJ_DG * q;
        if (i < w && c < w) *reinterpret_cast<float2 *>(Ao + 2 * ((size_t)(k0 + i) * ld + k0 + c)) = a[q];
    }
}

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2D tensor map (FP32 or FP16), 128-byte swizzle: `inner` elements per row,
// `rows` rows `row_bytes` apart, box of box_in elements x box_rows rows
bool tensor_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint64_t row_bytes,
                uint32_t box_in, uint32_t box_rows, bool half = false) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_in, box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(map, half ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base),
              dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

// pivot width of the outer Gauss-Jordan steps (the K of their products): 512
// by default, up to GJ_PMAX (a schedule choice of the autotuner)
constexpr int GJ_P = 512;
constexpr int GJ_PMAX = 1024;
// SMs the second part of each product (3) leaves free for the next pivot
// block's inverse, at pivot width 512 and 1024 (measured on the 21k cell's
// 16,790 block: at 1024, 8 / 12 / 16 / 24 / 32 / 48 SMs gave 47.0 / 46.0 /
// 44.9 / 44.2 / 43.6 / 46.6 ms per inversion; at 512, 4 / 16 gave 48.1 / 47.1)
#ifndef VIE_GJ_RESERVE_WIDE
#define VIE_GJ_RESERVE_WIDE 32
#endif
#ifndef VIE_GJ_RESERVE
#define VIE_GJ_RESERVE 16
#endif
static_assert(GJ_PMAX <= TC_KP, "the packed operands hold one outer pivot block");
static_assert(GJ_RQ == 32, "the row-publish jump covers 32 slots");
static_assert(GJ_W == 128 && GJ_P % GJ_W == 0 && GJ_PMAX % GJ_W == 0, "a pivot block is inverted in 128-wide steps");

constexpr int GJ_WORDS = 16;   // largest-entry words: 4 per set (products (a), (3)), 2 for the pivot blocks

size_t gj_pack_bytes(int n) {
    // two sets (consecutive outer steps overlap) of Ap [mp] and Bp [2 mp] FP16
    // rows, one set of 3 GJ_PMAX rows for the inversion of the pivot blocks, and
    // the largest-entry words of the packed operands
    const size_t mp = ((size_t)n + TC_TM - 1) / TC_TM * TC_TM;
    return (2 * 3 * mp + 3 * (size_t)GJ_PMAX) * TC_PACK_ROW * sizeof(__half) + GJ_WORDS * sizeof(unsigned);
}

namespace {
int tiles(int r, int c) { return ((r + TC_TM - 1) / TC_TM) * ((c + TC_TN - 1) / TC_TN); }
int kchunks(int w) { return (2 * w + TC_KCHUNK - 1) / TC_KCHUNK; }

// Packs the operands of one product from A (row stride ld): panel pa into Ap
// (mp rows, k_tc_pack_a) and panel pb, times sgn, into Bp (2 x 32 x bx rows,
// k_tc_pack_b), each scaled by the power of two its largest entry (found first
// into amax[0], amax[1]) selects.
void tc_pack(cudaStream_t st, const float *A, size_t ld, const TcPanel &pa, int mp, const TcPanel &pb, float sgn,
             int bx, unsigned *amax, __half *Ap, __half *Bp) {
    cudaMemsetAsync(amax, 0, 2 * sizeof(unsigned), st);
    const int big = std::max(pa.n1 * pa.w, pb.n1 * pb.w);
    const unsigned gx = (unsigned)std::max(1, std::min((big + 2047) / 2048, 2 * 152));
    k_tc_absmax<<<dim3(gx, 2), 256, 0, st>>>(A, ld, pa, pb, amax); ++g_launches;
    // only the K chunks the product reads: 32 complex K per chunk of 64 FP16
    const int kp = std::min(TC_KP, (std::max(pa.w, pb.w) + 31) / 32 * 32);
    k_tc_pack_a<<<(unsigned)(((size_t)mp * kp + 255) / 256), 256, 0, st>>>(A, ld, pa.n1, pa.c0, pa.w, pa.at, pa.skip,
                                                                          mp, kp, amax, Ap); ++g_launches;
    k_tc_pack_b<<<dim3(bx, kp / 32), 256, 0, st>>>(A, ld, pb.n1, pb.c0, pb.w, pb.at, pb.skip, sgn, amax + 1, Bp);
    ++g_launches;
}

// One tensor-core product on stream s with the maps of one operand set; timed
// (CUDA events; algorithmic bytes: read and write of the rows x cols block of
// C, one read of the two packed FP16 operand panels of width w; algorithmic
// flops 8 rows cols w) when kt is given.
void tc_product(cudaStream_t s, const CUtensorMap &tA, const CUtensorMap &tB, const CUtensorMap &tC,
                const CUtensorMap &tCs, const TcMap &mp, int grid, int *status, KernelTimer *kt, double rows,
                double cols, int w) {
    cudaEvent_t e0 = kt ? kt->next() : nullptr, e1 = kt ? kt->next() : nullptr;
    if (e0) cudaEventRecord(e0, s);
    k_tc_update<<<grid, TC_THREADS, TC_SMEM, s>>>(tA, tB, tC, tCs, mp, status); ++g_launches;
    if (e1) {
        cudaEventRecord(e1, s);
        // a complex multiply-add is 8 real flops: 8 rows cols w per product
        kt->add(e0, e1, 16.0 * rows * cols + 4.0 * (rows + cols) * w, 8.0 * rows * cols * w);
    }
}

// In-place inverse of the w x w pivot block at Ab (row stride ld, w <= GJ_PMAX):
// Gauss-Jordan with 128-wide pivots (register inverse of each 128 block, then
// its column-panel and trailing/row-panel products, K = 128).  sub: packed
// operand scratch of 3 GJ_PMAX rows; amax: two largest-entry words.
cudaError_t invert_pivot_block(float *Ab, size_t ld, int w, int *status, __half *sub, unsigned *amax, int sms,
                               cudaStream_t st) {
    k_gj_diag_w<<<1, GJ_W * GJ_DG, 0, st>>>(Ab, ld, 0, std::min(w, GJ_W), status); ++g_launches;
    if (w <= GJ_W) return cudaGetLastError();
    __half *Ap = sub, *Bp = sub + (size_t)GJ_PMAX * TC_PACK_ROW;
    const int wc = (w + 3) / 4 * 4;   // whole 16-byte column groups (padding columns stay zero)
    CUtensorMap tA, tB, tC, tCs;
    if (!tensor_map(&tA, Ap, TC_PACK_ROW, GJ_PMAX, TC_PACK_ROW * 2, TC_KCHUNK, TC_TM, true) ||
        !tensor_map(&tB, Bp, TC_PACK_ROW, 2 * (uint64_t)GJ_PMAX, TC_PACK_ROW * 2, TC_KCHUNK, 2 * TC_TN, true) ||
        !tensor_map(&tC, Ab, 2 * (uint64_t)wc, w, 8 * ld, 32, TC_TM) ||
        !tensor_map(&tCs, Ab, 2 * (uint64_t)wc, w, 8 * ld, 32, 32))
        return cudaErrorInvalidValue;
    const int wp = (w + TC_TM - 1) / TC_TM * TC_TM;
    for (int k1 = 0; k1 < w; k1 += GJ_W) {
        const int wi = std::min(GJ_W, w - k1), m1 = w - wi;
        if (k1 > 0) { k_gj_diag_w<<<1, GJ_W * GJ_DG, 0, st>>>(Ab, ld, k1, wi, status); ++g_launches; }
        const int mp1 = (m1 + TC_TM - 1) / TC_TM * TC_TM;
        tc_pack(st, Ab, ld, TcPanel{m1, k1, wi, k1, wi}, mp1, TcPanel{wi, k1, wi, 0, k1}, -1.f, TC_TN / 32, amax, Ap, Bp);
        tc_product(st, tA, tB, tC, tCs, TcMap{m1, wi, k1, wi, 0, k1, 0, 0, 1, 0, 0, 0, 0, kchunks(wi), amax},
                   std::min(tiles(m1, wi), sms), status, nullptr, 0, 0, 0);
        tc_pack(st, Ab, ld, TcPanel{w, k1, wi, w, 0}, wp, TcPanel{m1, k1, wi, k1, wi}, 1.f, mp1 / 32, amax, Ap, Bp);
        tc_product(st, tA, tB, tC, tCs, TcMap{w, m1, w, 0, k1, wi, k1 / TC_TM, 1, 0, 0, 0, 0, 0, kchunks(wi), amax},
                   std::min(tiles(w, m1), sms), status, nullptr, 0, 0, 0);
    }
    return cudaGetLastError();
}
}  // namespace

// One outer Gauss-Jordan step with pivot block P = A[k0:k0+w, k0:k0+w]
// (w = 512; rows and columns outside it: the trailing set T):
//   1. P <- P^-1                                  (invert_pivot_block)
//   2. A[T, P] <- -A[T, P] P^-1                   (product (a): trailing rows x pivot columns, beta 0)
//   3. A[T, T] <- A[T, T] + A[T, P] A[P, T],  A[P, T] <- P^-1 A[P, T]
//      as one product over all rows in natural order (the pivot rows' A operand
//      is P^-1) x the trailing columns, beta 0 on the pivot tile rows
// Products (a) and (3) run on the tensor cores from packed operands (K = 512:
// every step streams the whole n x (n - w) matrix, so the HBM traffic of the
// inversion is 16 n^3 / w bytes; at w = 512 the products sit near the ridge of
// the FP16 tensor rate and the HBM bandwidth).
// Look-ahead: product (3) is split into the tile columns holding the next
// pivot block (on st) and the rest (on aux, on all SMs but a reserve).  The next
// step's pivot inverse and column-panel product need only the first part, so
// they run on st while the rest of (3) streams through HBM; the next row-panel
// packing waits for it.  Consecutive steps use alternate packing buffers.
cudaError_t gj_invert_tc(float *A, size_t ld, int n, int *status, void *pack, cudaStream_t st, cudaStream_t aux,
                         KernelTimer *kt, int pivot) {
    const int P = (pivot == GJ_PMAX) ? GJ_PMAX : GJ_P;   // outer pivot width
    // SMs the rest of each product leaves to the next pivot block's inverse
    // (its K = 128 products; a 1024-wide block has eight 128-wide steps)
    const int reserve = P > GJ_P ? VIE_GJ_RESERVE_WIDE : VIE_GJ_RESERVE;
    int dev = 0, sms = 0;
    {   // opt in to the large dynamic shared memory (per device, cheap to repeat)
        cudaError_t e = cudaFuncSetAttribute(k_tc_update, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const int mpmax = (n + TC_TM - 1) / TC_TM * TC_TM;
    const size_t set_halves = 3 * (size_t)mpmax * TC_PACK_ROW;
    __half *const base = static_cast<__half *>(pack);
    __half *Ap[2], *Bp[2];
    __half *sub = base + 2 * set_halves;
    unsigned *words = reinterpret_cast<unsigned *>(sub + 3 * (size_t)GJ_PMAX * TC_PACK_ROW);   // GJ_WORDS
    CUtensorMap tmA[2], tmB[2], tmC, tmCs;
    for (int b = 0; b < 2; ++b) {
        Ap[b] = base + b * set_halves;
        Bp[b] = Ap[b] + (size_t)mpmax * TC_PACK_ROW;
    }
    if (n > P) {
        for (int b = 0; b < 2; ++b)
            if (!tensor_map(&tmA[b], Ap[b], TC_PACK_ROW, mpmax, TC_PACK_ROW * 2, TC_KCHUNK, TC_TM, true) ||
                !tensor_map(&tmB[b], Bp[b], TC_PACK_ROW, 2 * (uint64_t)mpmax, TC_PACK_ROW * 2, TC_KCHUNK, 2 * TC_TN,
                            true))
                return cudaErrorInvalidValue;
        if (!tensor_map(&tmC, A, 2 * (uint64_t)ld, n, 8 * ld, 32, TC_TM) ||
            !tensor_map(&tmCs, A, 2 * (uint64_t)ld, n, 8 * ld, 32, 32))
            return cudaErrorInvalidValue;
    }
    cudaEvent_t evP = nullptr, evB = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&evP, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&evB, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    bool pending = false;   // the second part of the previous product (3) is running on aux
    e = invert_pivot_block(A, ld, std::min(n, P), status, sub, words + 8, sms, st);
    for (int k0 = 0; k0 < n && e == cudaSuccess; k0 += P) {
        const int w = std::min(P, n - k0);
        const int m = n - w;
        if (m <= 0) break;
        const int cur = (k0 / P) & 1;
        const int mp = (m + TC_TM - 1) / TC_TM * TC_TM;
        const int kc = kchunks(w);
        unsigned *wa = words + 4 * cur, *w3 = wa + 2;   // this set's largest-entry words
        // (a) column panel: A[T, P] <- A[T, P] (-P^-1)
        tc_pack(st, A, ld, TcPanel{m, k0, w, k0, w}, mp, TcPanel{w, k0, w, 0, k0}, -1.f,
                (w + TC_TN - 1) / TC_TN * TC_TN / 32, wa, Ap[cur], Bp[cur]);
        tc_product(st, tmA[cur], tmB[cur], tmC, tmCs, TcMap{m, w, k0, w, 0, k0, 0, 0, 1, 0, 0, 0, 0, kc, wa},
                   std::min(tiles(m, w), sms), status, nullptr, 0, 0, 0);
        // (3) reads this step's row panel, which the previous step's second part wrote
        if (pending) { cudaStreamWaitEvent(st, evB, 0); pending = false; }
        tc_pack(st, A, ld, TcPanel{n, k0, w, n, 0}, mpmax, TcPanel{m, k0, w, k0, w}, 1.f, mp / 32, w3, Ap[cur], Bp[cur]);
        const int ntm = (n + TC_TM - 1) / TC_TM, nt = (m + TC_TN - 1) / TC_TN;
        const int prow = k0 / TC_TM, nprow = (w + TC_TM - 1) / TC_TM;   // pivot tile rows: beta 0
        const TcMap mb = {n, m, n, 0, k0, w, prow, nprow, 0, 0, 0, 0, 0, kc, w3};
        const bool next = k0 + P < n;
        const int tA = k0 / TC_TN, nA = std::min(P / TC_TN, nt - tA);   // tile columns of the next pivot block
        if (next && nt > nA) {
            TcMap ma = mb, mr = mb;
            ma.only_lo = tA; ma.only_n = nA;
            mr.skip_lo = tA; mr.skip_n = nA;
            const int colsA = std::min(nA * TC_TN, m - k0);
            tc_product(st, tmA[cur], tmB[cur], tmC, tmCs, ma, std::min(ntm * nA, sms), status, kt, n, colsA, w);
            cudaEventRecord(evP, st);
            cudaStreamWaitEvent(aux, evP, 0);
            tc_product(aux, tmA[cur], tmB[cur], tmC, tmCs, mr, std::max(1, std::min(ntm * (nt - nA), sms - reserve)),
                       status, kt, n, m - colsA, w);
            cudaEventRecord(evB, aux);
            pending = true;
        } else {
            tc_product(st, tmA[cur], tmB[cur], tmC, tmCs, mb, std::min(tiles(n, m), sms), status, kt, n, m, w);
        }
        if (next) {
            const int k1 = k0 + P;
            e = invert_pivot_block(A + 2 * ((size_t)k1 * ld + k1), ld, std::min(n - k1, P), status, sub, words + 8,
                                   sms, st);
        }
    }
    if (pending) cudaStreamWaitEvent(st, evB, 0);
    cudaEventDestroy(evP);
    cudaEventDestroy(evB);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// copy a diagonal block Z[off:off+n, off:off+n] into B (ld_b), converting precision
template <typename TS, typename TD>
__global__ void k_copy_block(const TS *Z, size_t ldz, int off, int n, TD *B, size_t ldb) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t tot = (size_t)n * ldb;
    if (e >= tot) return;
    int i = (int)(e / ldb), j = (int)(e % ldb);
    TD vr = 0, vi = 0;
    if (j < n) {
        vr = TD(Z[2 * ((size_t)(off + i) * ldz + off + j)]);
        vi = TD(Z[2 * ((size_t)(off + i) * ldz + off + j) + 1]);
    }
    B[2 * e] = vr;
    B[2 * e + 1] = vi;
}

template <typename TS, typename TD>
cudaError_t copy_block(const TS *Z, size_t ldz, int off, int n, TD *B, size_t ldb, cudaStream_t st) {
    size_t tot = (size_t)n * ldb;
    k_copy_block<TS, TD><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Z, ldz, off, n, B, ldb); ++g_launches;
    return cudaGetLastError();
}
template cudaError_t copy_block<float, float>(const float *, size_t, int, int, float *, size_t, cudaStream_t);
template cudaError_t copy_block<double, float>(const double *, size_t, int, int, float *, size_t, cudaStream_t);
template cudaError_t copy_block<double, double>(const double *, size_t, int, int, double *, size_t, cudaStream_t);

// ---------------------------------------------------------------------------
// GMRES vector kernels (two right-hand sides, [n][2] complex)
// ---------------------------------------------------------------------------
// h[j][r] += sum_i conj(V_j[i][r]) w[i][r]  for j < nv (atomics into FP64).
// Grid (chunks of DOT_CHUNK elements) x (vectors): every CTA streams one chunk
// of one basis vector with 16-byte loads, reduces in FP64 and adds 4 numbers.
constexpr int DOT_CHUNK = 2048;

__device__ __forceinline__ void load4(const float *p, double o[4]) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load4(const double *p, double o[4]) {
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

template <typename TV>
__global__ void __launch_bounds__(256) k_dots(const TV *V, size_t vstride, int nv, const TV *w, int n, double *h) {
    // FP32 vectors: FP32 products summed over a thread's 8 rows, FP64 from the
    // warp reduction on (the FP64 pipe is narrow); FP64 vectors: FP64 throughout
    using A = typename std::conditional<sizeof(TV) == 4, float, double>::type;
    __shared__ double red[8][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.y;
    const TV *v = V + (size_t)j * vstride;
    const int base = blockIdx.x * DOT_CHUNK;
    A a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
    for (int u = 0; u < DOT_CHUNK / 256; ++u) {
        const int i = base + u * 256 + threadIdx.x;
        if (i < n) {
            A x[4], y[4];
            if constexpr (sizeof(TV) == 4) {
                const float4 p = *reinterpret_cast<const float4 *>(v + 4 * (size_t)i);
                const float4 q = *reinterpret_cast<const float4 *>(w + 4 * (size_t)i);
                x[0] = p.x; x[1] = p.y; x[2] = p.z; x[3] = p.w;
                y[0] = q.x; y[1] = q.y; y[2] = q.z; y[3] = q.w;
            } else {
                double xd[4], yd[4];
                load4(v + 4 * (size_t)i, xd);
                load4(w + 4 * (size_t)i, yd);
                for (int c = 0; c < 4; ++c) { x[c] = xd[c]; y[c] = yd[c]; }
            }
            a0 += x[0] * y[0] + x[1] * y[1];
            a1 += x[0] * y[1] - x[1] * y[0];
            a2 += x[2] * y[2] + x[3] * y[3];
            a3 += x[2] * y[3] - x[3] * y[2];
        }
    }
    double d0 = a0, d1 = a1, d2 = a2, d3 = a3;
    for (int o = 16; o > 0; o >>= 1) {
        d0 += __shfl_down_sync(0xffffffffu, d0, o);
        d1 += __shfl_down_sync(0xffffffffu, d1, o);
        d2 += __shfl_down_sync(0xffffffffu, d2, o);
        d3 += __shfl_down_sync(0xffffffffu, d3, o);
    }
    if (lane == 0) { red[warp][0] = d0; red[warp][1] = d1; red[warp][2] = d2; red[warp][3] = d3; }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s2 = 0;
        for (int q = 0; q < 8; ++q) s2 += red[q][threadIdx.x];
        atomicAdd(h + 4 * j + threadIdx.x, s2);
    }
}

// w[i][r] -= sum_j V_j[i][r] h[j][r]   (h on the device, FP64)
// FP32 vectors: a CTA owns 32 rows (one per lane) and its 8 warps split the
// basis vectors; 16-byte loads, FP32 products and sums, the 8 partial sums
// combined through shared memory.  FP64 vectors: one thread per row.
__global__ void __launch_bounds__(256) k_subtract_f32(const float *V, size_t vstride, int nv, const double *h,
                                                      float *w, int n) {
    __shared__ float4 part[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    float s0r = 0.f, s0i = 0.f, s1r = 0.f, s1i = 0.f;
    if (i < n) {
#pragma unroll 2
        for (int j = warp; j < nv; j += 8) {
            const float4 v = *reinterpret_cast<const float4 *>(V + (size_t)j * vstride + 4 * (size_t)i);
            const double2 ha = __ldg(reinterpret_cast<const double2 *>(h + 4 * j));
            const double2 hb = __ldg(reinterpret_cast<const double2 *>(h + 4 * j + 2));
            const float h0 = (float)ha.x, h1 = (float)ha.y, h2 = (float)hb.x, h3 = (float)hb.y;
            s0r = fmaf(v.x, h0, fmaf(-v.y, h1, s0r));
            s0i = fmaf(v.x, h1, fmaf(v.y, h0, s0i));
            s1r = fmaf(v.z, h2, fmaf(-v.w, h3, s1r));
            s1i = fmaf(v.z, h3, fmaf(v.w, h2, s1i));
        }
    }
    part[warp][lane] = make_float4(s0r, s0i, s1r, s1i);
    __syncthreads();
    if (warp == 0 && i < n) {
        float4 t = part[0][lane];
        for (int q = 1; q < 8; ++q) {
            const float4 u = part[q][lane];
            t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
        }
        float4 *o = reinterpret_cast<float4 *>(w + 4 * (size_t)i);
        float4 c = *o;
        c.x -= t.x; c.y -= t.y; c.z -= t.z; c.w -= t.w;
        *o = c;
    }
}

template <typename TV>
__global__ void k_subtract(const TV *V, size_t vstride, int nv, const double *h, TV *w, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s0r = 0, s0i = 0, s1r = 0, s1i = 0;
    for (int j = 0; j < nv; ++j) {
        const TV *v = V + j * vstride + 4 * (size_t)i;
        const double *hh = h + 4 * j;
        s0r += double(v[0]) * hh[0] - double(v[1]) * hh[1];
        s0i += double(v[0]) * hh[1] + double(v[1]) * hh[0];
        s1r += double(v[2]) * hh[2] - double(v[3]) * hh[3];
        s1i += double(v[2]) * hh[3] + double(v[3]) * hh[2];
    }
    TV *o = w + 4 * (size_t)i;
    o[0] = TV(double(o[0]) - s0r);
    o[1] = TV(double(o[1]) - s0i);
    o[2] = TV(double(o[2]) - s1r);
    o[3] = TV(double(o[3]) - s1i);
}

// y[i][r] = s[r] * x[i][r] (complex scale per rhs; s on the host)
template <typename TX, typename TY>
__global__ void k_scale(const TX *x, TY *y, int n, double s0r, double s0i, double s1r, double s1i) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const TX *a = x + 4 * (size_t)i;
    TY *o = y + 4 * (size_t)i;
    double xr0 = a[0], xi0 = a[1], xr1 = a[2], xi1 = a[3];
    o[0] = TY(s0r * xr0 - s0i * xi0);
    o[1] = TY(s0r * xi0 + s0i * xr0);
    o[2] = TY(s1r * xr1 - s1i * xi1);
    o[3] = TY(s1r * xi1 + s1i * xr1);
}

// x[i][r] += sum_j V_j[i][r] y[j][r]  (y on the device)
template <typename TV>
__global__ void k_combine(const TV *V, size_t vstride, int nv, const double *y, double *x, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s0r = 0, s0i = 0, s1r = 0, s1i = 0;
    for (int j = 0; j < nv; ++j) {
        const TV *v = V + j * vstride + 4 * (size_t)i;
        const double *yy = y + 4 * j;
        s0r += double(v[0]) * yy[0] - double(v[1]) * yy[1];
        s0i += double(v[0]) * yy[1] + double(v[1]) * yy[0];
        s1r += double(v[2]) * yy[2] - double(v[3]) * yy[3];
        s1i += double(v[2]) * yy[3] + double(v[3]) * yy[2];
    }
    double *o = x + 4 * (size_t)i;
    o[0] += s0r; o[1] += s0i; o[2] += s1r; o[3] += s1i;
}

template <typename TV>
cudaError_t dots(const TV *V, size_t vstride, int nv, const TV *w, int n, double *h, cudaStream_t st) {
    if (nv <= 0 || n <= 0) return cudaSuccess;
    cudaMemsetAsync(h, 0, sizeof(double) * 4 * nv, st);
    k_dots<TV><<<dim3((n + DOT_CHUNK - 1) / DOT_CHUNK, nv), 256, 0, st>>>(V, vstride, nv, w, n, h); ++g_launches;
    return cudaGetLastError();
}
template <typename TV>
cudaError_t subtract(const TV *V, size_t vstride, int nv, const double *h, TV *w, int n, cudaStream_t st) {
    if constexpr (sizeof(TV) == 4) {
        k_subtract_f32<<<(n + 31) / 32, 256, 0, st>>>(V, vstride, nv, h, w, n);
    } else {
        k_subtract<TV><<<(n + 255) / 256, 256, 0, st>>>(V, vstride, nv, h, w, n);
    }
    ++g_launches;
    return cudaGetLastError();
}
template <typename TX, typename TY>
cudaError_t scale(const TX *x, TY *y, int n, const double s[4], cudaStream_t st) {
    k_scale<TX, TY><<<(n + 255) / 256, 256, 0, st>>>(x, y, n, s[0], s[1], s[2], s[3]); ++g_launches;
    return cudaGetLastError();
}
template <typename TV>
cudaError_t combine(const TV *V, size_t vstride, int nv, const double *y, double *x, int n, cudaStream_t st) {
    k_combine<TV><<<(n + 255) / 256, 256, 0, st>>>(V, vstride, nv, y, x, n); ++g_launches;
    return cudaGetLastError();
}
template cudaError_t dots<float>(const float *, size_t, int, const float *, int, double *, cudaStream_t);
template cudaError_t dots<double>(const double *, size_t, int, const double *, int, double *, cudaStream_t);
template cudaError_t subtract<float>(const float *, size_t, int, const double *, float *, int, cudaStream_t);
template cudaError_t subtract<double>(const double *, size_t, int, const double *, double *, int, cudaStream_t);
template cudaError_t scale<double, float>(const double *, float *, int, const double *, cudaStream_t);
template cudaError_t scale<float, float>(const float *, float *, int, const double *, cudaStream_t);
template cudaError_t scale<double, double>(const double *, double *, int, const double *, cudaStream_t);
template cudaError_t combine<float>(const float *, size_t, int, const double *, double *, int, cudaStream_t);
template cudaError_t combine<double>(const double *, size_t, int, const double *, double *, int, cudaStream_t);

}  // namespace vie
