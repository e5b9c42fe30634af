// Device-side pieces shared by the state-sweep kernels: the gate program,
// gate tensors built from angles (K0, fused into every consumer), and the
// per-amplitude gate actions.
//
// A sweep program is the state-sweep contraction path of the circuit's
// tensor network (Sec. 3.2 (e)): every gate tensor is absorbed, in circuit
// order, into the rank-n ket tensor psi[x], x = sum_q b_q 2^(n-1-q).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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

// Absorb one gate tensor (or its adjoint) into the tile.
__device__ __forceinline__ void tile_apply(c2* st, const SweepOp& op, const float* ang,
                                           const TileCtx& c, bool dag) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const uint32_t nloc = 1u << c.k;
  const int kind = op.kind;
  if (kind == K_CNOT) {
    const int lt = c.loc[op.p1], lc = c.loc[op.p0];
    if (lc >= 0) {
      const int lo = min(lc, lt), hi = max(lc, lt);
      for (uint32_t i = tid; i < (nloc >> 2); i += nt) {
        const uint32_t x = insert0(insert0(i, lo), hi) | (1u << lc);
        const c2 u = st[x], v = st[x | (1u << lt)];
        st[x] = v;
        st[x | (1u << lt)] = u;
      }
    } else if ((c.base >> op.p0) & 1u) {
      for (uint32_t i = tid; i < (nloc >> 1); i += nt) {
        const uint32_t x = insert0(i, lt);
        const c2 u = st[x], v = st[x | (1u << lt)];
        st[x] = v;
        st[x | (1u << lt)] = u;
      }
    }
  } else if (kind == K_CZ) {
    const int la = c.loc[op.p0], lb = c.loc[op.p1];
    if (la < 0 && !((c.base >> op.p0) & 1u)) return;
    if (lb < 0 && !((c.base >> op.p1) & 1u)) return;
    for (uint32_t x = tid; x < nloc; x += nt) {
      if (tbit(c, op.p0, x) & tbit(c, op.p1, x)) {
        const c2 u = st[x];
        st[x] = {-u.x, -u.y};
      }
    }
  } else if (kind == K_RZZ) {
    float s, co;
    sincosf(0.5f * ang[0], &s, &co);
    if (dag) s = -s;
    const c2 even = {co, -s}, odd = {co, s};
    for (uint32_t x = tid; x < nloc; x += nt)
      st[x] = cmul((tbit(c, op.p0, x) ^ tbit(c, op.p1, x)) ? odd : even, st[x]);
  } else if (is_diag_1q(kind)) {
    M2 m = gate_1q(kind, ang);
    if (dag) m = dagger(m);
    for (uint32_t x = tid; x < nloc; x += nt) st[x] = cmul(tbit(c, op.p0, x) ? m.m11 : m.m00, st[x]);
  } else {
    M2 m = gate_1q(kind, ang);
    if (dag) m = dagger(m);
    const int p = c.loc[op.p0];
    for (uint32_t i = tid; i < (nloc >> 1); i += nt) {
      const uint32_t x0 = insert0(i, p), x1 = x0 | (1u << p);
      c2 a0 = st[x0], a1 = st[x1];
      apply2(m, a0, a1);
      st[x0] = a0;
      st[x1] = a1;
    }
  }
}

// One step of the reverse sweep for gate `op` on a tile: un-compute psi,
// add the gate's angle derivatives of F into g[0..2] (this thread's share),
// propagate lambda.  psi and lambda enter as psi_g = G psi_{g-1} and
// lambda_g = (G_{g+1}..G_last)^dagger O psi_last.
//   Pauli rotations exp(-i t P/2): dF/dt = Im <lambda_g| P |psi_g>
//   U3: d/dtheta = 2 Re <lambda_g| dG/dtheta |psi_{g-1}>,
//       d/dphi = -2 Im(conj(lambda_g[1]) psi_g[1]),
//       d/dlambda = -2 Im(conj(lambda_{g-1}[1]) psi_{g-1}[1]).
__device__ __forceinline__ void tile_adjoint(c2* psi, c2* lam, const SweepOp& op,
                                             const float* ang, const TileCtx& c, float* g) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const uint32_t nloc = 1u << c.k;
  const int kind = op.kind;
  if (kind == K_CNOT || kind == K_CZ) {  // self-inverse, no angles
    tile_apply(psi, op, ang, c, true);
    tile_apply(lam, op, ang, c, true);
    return;
  }
  if (kind == K_RZZ || is_diag_1q(kind)) {
    float s, co;
    sincosf(0.5f * ang[0], &s, &co);
    float acc = 0.f;
    for (uint32_t x = tid; x < nloc; x += nt) {
      const int bit = (kind == K_RZZ) ? (tbit(c, op.p0, x) ^ tbit(c, op.p1, x)) : tbit(c, op.p0, x);
      const float sg = bit ? -1.f : 1.f;
      const c2 p = psi[x], l = lam[x];
      acc += sg * (l.x * p.y - l.y * p.x);  // s(x) Im(conj(l) p)
      c2 dd;                                 // conj of the diagonal entry
      if (kind == K_Z) dd = {sg, 0.f};
      else dd = {co, bit ? -s : s};
      psi[x] = cmul(dd, p);
      lam[x] = cmul(dd, l);
    }
    g[0] += acc;
    return;
  }
  const M2 md = dagger(gate_1q(kind, ang));
  M2 dth{};
  if (kind == K_U3) dth = u3_dtheta(ang);
  const int p = c.loc[op.p0];
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  for (uint32_t i = tid; i < (nloc >> 1); i += nt) {
    const uint32_t x0 = insert0(i, p), x1 = x0 | (1u << p);
    c2 p0 = psi[x0], p1 = psi[x1], l0 = lam[x0], l1 = lam[x1];
    if (kind == K_RX) {
      a0 += (l0.x * p1.y - l0.y * p1.x) + (l1.x * p0.y - l1.y * p0.x);
    } else if (kind == K_RY) {
      a0 += -(l0.x * p1.x + l0.y * p1.y) + (l1.x * p0.x + l1.y * p0.y);
    } else if (kind == K_U3) {
      a1 += -2.f * (l1.x * p1.y - l1.y * p1.x);
    }
    apply2(md, p0, p1);
    if (kind == K_U3) {
      c2 d0 = p0, d1 = p1;
      apply2(dth, d0, d1);
      const c2 z = cadd(cmulc(l0, d0), cmulc(l1, d1));
      a0 += 2.f * z.x;
    }
    apply2(md, l0, l1);
    if (kind == K_U3) a2 += -2.f * (l1.x * p1.y - l1.y * p1.x);
    psi[x0] = p0;
    psi[x1] = p1;
    lam[x0] = l0;
    lam[x1] = l1;
  }
  g[0] += a0;
  g[1] += a1;
  g[2] += a2;
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
  for (int j = 0; j < op.nang; j++) ang[j] = op_angle(op, j, a.params, a.pstride, a.inputs, a.F, b, bad);
  if (k > 0) {
    const int e = (k - 1) >> 1;
    if (a.ps_gate[e] == gi) ang[a.ps_ang[e]] += ((k - 1) & 1) ? -kHalfPiF : kHalfPiF;
  }
}

}  // namespace tdq
