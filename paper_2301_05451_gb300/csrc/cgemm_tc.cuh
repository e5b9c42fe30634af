// K3: complex batched "NT" product on the 5th-generation tensor cores.
//
//   D[i][j] = sum_k X[i][k] Y[j][k]      (complex64, both operands k-contiguous)
//
// in 3xTF32 split precision: every FP32 operand is written as hi + lo with
// hi = tf32(x) and lo = tf32(x - hi), and each real product is taken as
// hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding), accumulated
// in FP32 in tensor memory.  A complex product needs the four real products
// Xr Yr, Xi Yi, Xr Yi, Xi Yr; Re D = Xr Yr - Xi Yi is kept as two accumulators
// (added and subtracted in the epilogue), Im D as one.
//
// One CTA computes a 128 x 64 tile of D, warp-specialised: sixteen converter
// warps stream k-blocks of X and Y through a cp.async ring, split them into
// TF32 hi / lo planes in one of four shared-memory stages and arrive on the
// stage's "full" mbarrier; one issuer thread waits on it, issues the
// tcgen05.mma instructions (M = 128, N = 64, K = 8 TF32 each) and commits to
// the stage's "empty" mbarrier.  The accumulators (6 x 64 columns of 128
// lanes) live in TMEM; every 16 k-blocks the converters read them out with
// tcgen05.ld into FP32 sums (the tensor cores' FP32 accumulation rounds toward
// zero; the sums round to nearest).  No CTA-wide barrier in the main loop.
// Every wait is bounded: on a timeout the kernel sets an error bit, waits
// (bounded) for the products in flight, frees its TMEM and returns.
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
