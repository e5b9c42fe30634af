// K3: complex batched "NT" product on the 5th-generation tensor cores.
//
//   D[i][j] = sum_k X[i][k] Y[j][k]      (complex64, both operands k-contiguous)
//
// in 3xTF32 split precision: every FP32 operand is written as hi + lo with
// hi = tf32(x) and lo = tf32(x - hi), and each real product is taken as
// hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding), accumulated
// in FP32 in tensor memory.  The complex product is computed as one real
// product of the embedding [Xr Xi] [[Yr Yi]; [-Yi Yr]]^T, whose output
// columns are Re D and Im D side by side; with the hi and lo planes of Y
// stacked, a k-block of 8 complex takes four tcgen05.mma instructions (M 128,
// K 8 TF32; N 256, 128, 256, 128) instead of twelve of N 64.
//
// One CTA computes a 128 x 64 tile of D, warp-specialised and converged per
// warp: a TMA producer streams pairs of k-blocks of X and Y into a raw ring
// (128-byte swizzle); sixteen converter warps split them into TF32 hi / lo
// planes -- X's into one of four TMEM stages (tcgen05.st), where the products
// read their A operand, Y's into one of four shared-memory stages -- and
// arrive on the stage's "full" mbarrier; the issuer warp waits on it, one
// lane issues the products and commits to the stage's "empty" mbarrier.
// TMEM also holds the hi*hi terms of the current 16-k-block chunk in one of
// two alternating 128-column buffers and the hi*lo + lo*hi corrections of the
// whole K; four flusher warps add each finished chunk into FP32 sums in
// shared memory with round-to-nearest adds (the tensor cores' FP32
// accumulation rounds toward zero) while the next chunk accumulates.  The
// epilogue stages the finished tile in shared memory and writes whole rows.
// No CTA-wide barrier in the main loop.  Every wait is bounded: on a timeout
// the kernel sets an error bit, waits (bounded) for the products and copies
// in flight, frees its TMEM and returns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tdq {

// Epilogue index map: D[i][j] goes to out[ scatter(i) | scatter(j) ] where the
// bits of i and j are deposited at the given positions (or row-major when
// rowmajor_ld > 0: out[i * ld + j]).
struct CgemmOut {
  const int8_t* ipos;  // bit position of i bit b (nullptr with rowmajor)
  const int8_t* jpos;
  int ni, nj;          // bits of i and j
  int64_t ld;          // > 0: row-major with this leading dimension
};

// Bound (ns of the global timer) of every wait of the main loop; the wait
// for the products in flight at the end keeps this bound whatever the
// caller asks for the main loop.
constexpr int64_t kCgemmWaitNs = 1000000000ll;

// Launch D = X Y^T for `batch` independent problems (strides in complex
// elements).  X: [I][K], Y: [J][K], I % 128 == 0, J % 64 == 0, K % 8 == 0.
// wait_ns bounds each wait of the main loop (the stage, chunk and read-out
// handshakes).  Returns cudaSuccess or an error; *where (if given) names the
// failing stage.
cudaError_t cgemm_tc_launch(const float2* X, int64_t xs, const float2* Y, int64_t ys, float2* out, int64_t os,
                            int I, int J, int K, int batch, const CgemmOut& map, int* status, cudaStream_t st,
                            const char** where = nullptr, int64_t wait_ns = kCgemmWaitNs);

}  // namespace tdq
