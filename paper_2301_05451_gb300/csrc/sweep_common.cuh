// Device-side pieces shared by the state-sweep kernels: the gate program,
// gate tensors built from angles (K0, fused into every consumer), and the
// per-amplitude gate actions.
//
// A sweep program is the state-sweep contraction path of the circuit's
// tensor network (Sec. 3.2 (e)): every gate tensor is absorbed, in circuit
// order, into the rank-n ket tensor psi[x], x = sum_q b_q 2^(n-1-q).
#pragma once

#ifdef __CUDACC_RTC__
// run-time compilation (specialised programs): no host headers
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef short int16_t;
typedef unsigned short uint16_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef long long int64_t;
typedef unsigned long long uint64_t;
#else
#include <cuda_runtime.h>
#include <stdint.h>
#endif

#include "tdq.h"

namespace tdq {

enum : int {
  K_H = 0, K_X = 1, K_Y = 2, K_Z = 3, K_RX = 4, K_RY = 5, K_RZ = 6, K_U3 = 7,
  K_CNOT = 8, K_CZ = 9, K_RZZ = 10
};

// One gate of the device program.  Bit positions, not qubit numbers.
struct SweepOp {
  int8_t kind;
  int8_t p0;       // bit position of the first qubit (control for CNOT)
  int8_t p1;       // bit position of the second qubit, -1 for 1-qubit gates
  int8_t nang;
  int32_t src[3];  // >= 0 parameter column, -1 fixed, <= -2 input (-2 - j)
  float fixed[3];
  int32_t slot[3]; // parameter column receiving the gradient, or -1
};

struct c2 {
  float x, y;
};

__device__ __forceinline__ c2 cmul(c2 a, c2 b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ c2 cadd(c2 a, c2 b) { return {a.x + b.x, a.y + b.y}; }
// conj(a) * b
__device__ __forceinline__ c2 cmulc(c2 a, c2 b) { return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; }
__device__ __forceinline__ c2 cfma(c2 a, c2 b, c2 acc) {
  return {fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y))};
}

// 2x2 matrix [[m00, m01], [m10, m11]] acting as (a0, a1) -> (m00 a0 + m01 a1, m10 a0 + m11 a1)
struct M2 {
  c2 m00, m01, m10, m11;
};

__device__ __forceinline__ M2 dagger(const M2& m) {
  return {{m.m00.x, -m.m00.y}, {m.m10.x, -m.m10.y}, {m.m01.x, -m.m01.y}, {m.m11.x, -m.m11.y}};
}

__device__ __forceinline__ void apply2(const M2& m, c2& a0, c2& a1) {
  c2 b0 = cfma(m.m01, a1, cmul(m.m00, a0));
  c2 b1 = cfma(m.m11, a1, cmul(m.m10, a0));
  a0 = b0;
  a1 = b1;
}

// Angle j of op for row b; flags non-finite values in *bad.
__device__ __forceinline__ float op_angle(const SweepOp& op, int j, const float* params,
                                          int64_t pstride, const float* inputs, int F, int64_t b,
                                          int* bad) {
  const int s = op.src[j];
  float v;
  if (s >= 0) v = params[b * pstride + s];
  else if (s == -1) v = op.fixed[j];
  else v = inputs[b * F + (-2 - s)];
  if (!isfinite(v)) *bad = 1;
  return v;
}

// The 2x2 tensor of a one-qubit gate (gate conventions of the C ABI header).
__device__ __forceinline__ M2 gate_1q(int kind, const float* a) {
  const float r = 0.70710678118654752f;
  float s, c;
  switch (kind) {
    case K_H: return {{r, 0}, {r, 0}, {r, 0}, {-r, 0}};
    case K_X: return {{0, 0}, {1, 0}, {1, 0}, {0, 0}};
    case K_Y: return {{0, 0}, {0, -1}, {0, 1}, {0, 0}};
    case K_Z: return {{1, 0}, {0, 0}, {0, 0}, {-1, 0}};
    case K_RX:
      sincosf(0.5f * a[0], &s, &c);
      return {{c, 0}, {0, -s}, {0, -s}, {c, 0}};
    case K_RY:
      sincosf(0.5f * a[0], &s, &c);
      return {{c, 0}, {-s, 0}, {s, 0}, {c, 0}};
    case K_RZ:
      sincosf(0.5f * a[0], &s, &c);
      return {{c, -s}, {0, 0}, {0, 0}, {c, s}};
    default: {  // K_U3
      float sp, cp, sl, cl, spl, cpl;
      sincosf(0.5f * a[0], &s, &c);
      sincosf(a[1], &sp, &cp);
      sincosf(a[2], &sl, &cl);
      sincosf(a[1] + a[2], &spl, &cpl);
      return {{c, 0}, {-cl * s, -sl * s}, {cp * s, sp * s}, {cpl * c, spl * c}};
    }
  }
}

// dU3/dtheta
__device__ __forceinline__ M2 u3_dtheta(const float* a) {
  float s, c, sp, cp, sl, cl, spl, cpl;
  sincosf(0.5f * a[0], &s, &c);
  sincosf(a[1], &sp, &cp);
  sincosf(a[2], &sl, &cl);
  sincosf(a[1] + a[2], &spl, &cpl);
  return {{-0.5f * s, 0}, {-0.5f * cl * c, -0.5f * sl * c}, {0.5f * cp * c, 0.5f * sp * c},
          {-0.5f * cpl * s, -0.5f * spl * s}};
}

__device__ __forceinline__ bool is_diag_1q(int kind) { return kind == K_RZ || kind == K_Z; }

// insert a zero bit at position p of i
__device__ __forceinline__ uint32_t insert0(uint32_t i, int p) {
  const uint32_t lo = i & ((1u << p) - 1u);
  return ((i >> p) << (p + 1)) | lo;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Observable terms: position mask of Z's, coefficient, group (sorted by group).
struct TermDev {
  uint32_t pmask_lo, pmask_hi;
  float coeff;
  int group;
};

// sum_{t in [t0, t1)} coeff_t * (-1)^{popc(x & mask_t)}: the diagonal of a
// group of Z-product terms at basis index x.
__device__ __forceinline__ float diag_weight(const TermDev* terms, int t0, int t1, uint32_t x) {
  float d = 0.f;
  for (int t = t0; t < t1; t++) d += (__popc(x & terms[t].pmask_lo) & 1) ? -terms[t].coeff : terms[t].coeff;
  return d;
}

struct SweepArgs {
  const SweepOp* ops;
  int G, n;
  const float* params;
  int64_t pstride;
  const float* inputs;
  int F;
  const TermDev* terms;
  const int* group_ptr;  // terms of group g: [group_ptr[g], group_ptr[g+1])
  int T, n_groups;
  const uint32_t* amp_idx;
  int A, output;
  double* values;
  const double* gw;
  float* grads;
  int P;
  int* status;
  // parameter shift: row r is (b, k) = (r / ps_copies, r % ps_copies); k = 0
  // unshifted, k = 2j+1 / 2j+2 has angle j shifted by +pi/2 / -pi/2
  int ps_copies;
  const int* ps_gate;
  const int* ps_ang;
  double* ps_F;
  // diagonal of each output group's observable, [n_groups][2^n], or NULL
  const float* odiag;
  // initial state of row b: init + b * init_stride (NULL: |0...0>)
  const c2* init;
  int64_t init_stride;
};

// One circuit of a multi-circuit launch: its sweep arguments with the
// per-call pointers left NULL, its gate-tensor recipes, and the offsets
// (elements) of its rows in the packed parameter, input, value, weight and
// gradient buffers.
struct MultiCirc {
  SweepArgs a;
  const int* rec_ptr;
  const int* rec_ops;
  int nrec;
  int64_t p_off, x_off, v_off, g_off;
};

// A tile of the state in shared memory: local element j holds the amplitude
// at the global index whose bits in the tile's positions are j's bits
// (position p is local bit loc[p]) and whose other bits are those of base.
struct TileCtx {
  const int8_t* loc;
  uint32_t base;
  int k;
};

__device__ __forceinline__ int tbit(const TileCtx& c, int p, uint32_t j) {
  const int l = c.loc[p];
  return l >= 0 ? (int)((j >> l) & 1u) : (int)((c.base >> p) & 1u);
}

// Block-wide double sum (blockDim a multiple of 32); every thread gets it.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum_d(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; i++) t += red[i];
  return t;
}

constexpr float kHalfPiF = 1.57079632679489661923f;

// Angles of op for row (b, shift copy k).
__device__ __forceinline__ void row_angles(const SweepArgs& a, const SweepOp& op, int gi, int64_t b,
                                           int k, float* ang, int* bad) {
  int sa = -1;
  float sh = 0.f;
  if (k > 0) {
    const int e = (k - 1) >> 1;
    if (a.ps_gate[e] == gi) {
      sa = a.ps_ang[e];
      sh = ((k - 1) & 1) ? -kHalfPiF : kHalfPiF;
    }
  }
#pragma unroll
  for (int j = 0; j < 3; j++)
    if (j < op.nang) ang[j] = op_angle(op, j, a.params, a.pstride, a.inputs, a.F, b, bad) + (j == sa ? sh : 0.f);
}

}  // namespace tdq
