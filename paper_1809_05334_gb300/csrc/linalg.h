// Dense complex linear algebra used by the solve (see linalg.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <utility>
#include <vector>

#include "vie_internal.h"

namespace vie {

// y <- alpha Z x (+ y if accumulate) for FP32 Z and FP64 x, y, at double-length
// accuracy from FP32 arithmetic (x split into two FP32 parts, exact products,
// compensated sums); xs is device scratch of 8 cols floats
cudaError_t matvec_ds(const float *A, size_t ld, int rows, int cols, const double *x, float *xs, double *y,
                      double alpha, bool accumulate, cudaStream_t st);
// y <- alpha A x (+ y if accumulate) for two right-hand sides; grid_mult: row
// ranges per resident CTA (1: one; the autotuner may pick more)
template <typename TZ, typename TX, typename TA>
cudaError_t matvec(const TZ *A, size_t ld, int rows, int cols, const TX *x, TA *y, TA alpha, bool accumulate,
                   cudaStream_t st, int grid_mult = 1);
// CUDA-event timing of selected launches (optional)
struct KernelTimer {
    cudaEvent_t (*alloc)(void *) = nullptr;   // returns the next event of the caller's pool
    void *pool = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    std::vector<double> work;    // algorithmic bytes of each timed launch
    std::vector<double> flops;   // and its algorithmic flops
    cudaEvent_t next() { return alloc ? alloc(pool) : nullptr; }
    void add(cudaEvent_t a, cudaEvent_t b, double w, double f = 0) {
        ev.push_back({a, b});
        work.push_back(w);
        flops.push_back(f);
    }
};
// In-place inversion of an n x n complex FP32 block (no pivoting) by blocked
// Gauss-Jordan with 512-wide outer pivot blocks and the tcgen05 products
// (FP16 operands with power-of-two scales, FP32 accumulation); *status gets
// bit 0 for a zero or non-finite pivot and bit 1 for a bounded device wait
// that ran out;
// `pack` is device scratch of gj_pack_bytes(n) bytes (the packed operands and
// their scale words), aux a second stream of the caller (look-ahead); the work
// is complete on st when the last call returns on it
size_t gj_pack_bytes(int n);
// pivot: width of the outer pivot blocks, 512 (default) or 1024 (half the
// passes over the block, a longer chain of pivot-block inverses)
cudaError_t gj_invert_tc(float *A, size_t ld, int n, int *status, void *pack, cudaStream_t st, cudaStream_t aux,
                         KernelTimer *kt = nullptr, int pivot = 512);
// one bounded mbarrier wait of at most `polls` polls on a barrier that gets its
// arrival (arrive) or never does: bit 1 of *status (device) when it runs out
cudaError_t wait_check(bool arrive, long long polls, int *status, cudaStream_t st);
// one launch of the FMA-loop peak kernel (FP32 or FP64), events e0/e1 around
// it on st; *flops = its floating-point operations
cudaError_t fma_peak(bool fp64, int iters, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, double *flops);
// *out (zeroed by the caller) <- max |A[i]| over count floats, as float bits
cudaError_t absmax(const float *A, size_t count, unsigned *out, cudaStream_t st);
// 16-bit copies of complex FP32 matrices in the column-interleaved layout the
// 16-bit products read: rows of ld16(cols) complex entries; inside each chunk
// of 128 columns, position p holds column (p % 4) * 32 + p / 4 of the chunk
// (zero past cols), so the four entries of one 16-byte load are columns
// j, j + 32, j + 64, j + 96 and the product's x loads are contiguous across a
// warp.  il_pos(c): the position of column c.
inline size_t ld16(int cols) { return ((size_t)cols + 127) / 128 * 128; }
__host__ __device__ inline size_t il_pos(size_t c) {
    const size_t j = c & 127;
    return (c - j) + (j & 31) * 4 + (j >> 5);
}
// B = scale A in FP16 (interleaved; A: rows x cols complex, row stride lda complex)
cudaError_t to_half_il(const float *A, size_t lda, int rows, int cols, float scale, __half *B, cudaStream_t st);
// B = A in BF16 (interleaved)
cudaError_t to_bf16_il(const float *A, size_t lda, int rows, int cols, __nv_bfloat16 *B, cudaStream_t st);
template <typename TS, typename TD>
cudaError_t copy_block(const TS *Z, size_t ldz, int off, int n, TD *B, size_t ldb, cudaStream_t st);
template <typename TV>
cudaError_t dots(const TV *V, size_t vstride, int nv, const TV *w, int n, double *h, cudaStream_t st);
template <typename TV>
cudaError_t subtract(const TV *V, size_t vstride, int nv, const double *h, TV *w, int n, cudaStream_t st);
template <typename TX, typename TY>
cudaError_t scale(const TX *x, TY *y, int n, const double s[4], cudaStream_t st);
template <typename TV>
cudaError_t combine(const TV *V, size_t vstride, int nv, const double *y, double *x, int n, cudaStream_t st);

}  // namespace vie
