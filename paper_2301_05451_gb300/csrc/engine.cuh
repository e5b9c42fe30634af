// Register-pass gate absorption: the inner engine of the sweep kernels.
//
// A tile of 2^k amplitudes sits in shared memory (swizzled, see swz).  Its
// gate program is cut into register passes: a pass names M <= 4 tile-local
// bits; each thread loads one group of 2^M amplitudes that differ only in
// those bits into registers, absorbs every gate of the pass there, and stores
// the group back.  A gate fits a pass when its non-diagonal target bits are
// among the M bits; diagonal gates (RZ, Z, CZ, RZZ) and CNOT controls read
// any other bit from the group's index (or from the bits fixed for the tile).
// One shared-memory sweep then carries many gates instead of one.
#pragma once

#include "sweep_common.cuh"

namespace tdq {

constexpr int kMaxRegBits = 4;
// register bits of forward (fused) and reverse (per-gate) programs: generic
// and tiled programs, and whole-state programs specialised to a circuit
constexpr int kFwdRegBits = 4;
constexpr int kRevRegBits = 3;
constexpr int kSpecFwdRegBits = 2;
constexpr int kSpecRevRegBits = 2;
// tiled programs specialised to the circuit: their passes stream the state
// through HBM, and wide register passes mean fewer shared-memory round trips
// (the 20-qubit ladder: 4/4 bits 4715 evals/s against 4536 at 4/3 and 4407
// at 3/3, GB300)
constexpr int kTiledSpecFwdRegBits = 4;
constexpr int kTiledSpecRevRegBits = 4;
// Gradient slots at most per reverse register pass (its accumulators live in
// registers beside the pass's amplitudes; the 20-qubit ladder's reverse
// passes spilled registers with 20 and more)
#ifndef TDQ_REV_PASS_SLOTS
#define TDQ_REV_PASS_SLOTS 8
#endif
constexpr int kRevPassSlots = TDQ_REV_PASS_SLOTS;

struct RegPass {
  int8_t m;          // register bits (1..4)
  int8_t lb[4];      // tile-local bit indices, ascending
  int32_t op_begin;  // decoded ops [op_begin, op_end) of the program
  int32_t op_end;
};

constexpr int K_FUSED = 11;  // product of consecutive one-qubit gates on one qubit

// A gate decoded for one register pass (built on the host).
struct DOp {
  uint8_t kind;     // gate kind or K_FUSED
  int8_t r0, r1;    // register bit holding position p0 / p1, or -1
  int8_t l0, l1;    // else: tile-local bit giving the value, or -1 (fixed for the tile)
  int8_t p0, p1;    // global bit positions
  uint8_t nang;     // angles with gradients (reverse programs)
  int16_t slot[3];  // gradient slot of each angle, or -1
  int16_t mat;      // row of the per-row gate-tensor table
};
static_assert(sizeof(DOp) == 16, "DOp layout");

// Bank-conflict-free shared-memory index of tile element x (8-byte
// elements): the low 4 bits are XORed with bits 4..7.  A bijection.
__device__ __forceinline__ uint32_t swz(uint32_t x) { return x ^ ((x >> 4) & 15u); }

// Gate tensor of op o for one row: forward matrix (diagonal gates keep their
// two phases in m00 / m11), and for U3 dU3/dtheta.
struct OpMat {
  M2 m;
  M2 d;
};

__device__ __forceinline__ OpMat build_opmat(const SweepOp& op, const float* ang) {
  OpMat r{};
  switch (op.kind) {
    case K_CNOT: case K_CZ: break;
    case K_RZZ: {
      float s, c;
      sincosf(0.5f * ang[0], &s, &c);
      r.m.m00 = {c, -s};  // even parity: e^{-i t/2}
      r.m.m11 = {c, s};   // odd parity:  e^{+i t/2}
      break;
    }
    default:
      r.m = gate_1q(op.kind, ang);
      if (op.kind == K_U3) r.d = u3_dtheta(ang);
  }
  return r;
}

// ------------------------------------------------------ packed FP32x2 arithmetic
// A complex amplitude's (re, im) halves sit in one 64-bit register pair, and
// the sm_100-family packed instructions (__ffma2_rn, __fmul2_rn) work on both
// halves at once: one issue slot for two FP32 operations.  Real rotations
// and the gradient dot products pack directly; a complex coefficient m
// multiplies as m a = (m.x, m.x) . a + (-m.y, m.y) . (a.y, a.x).
__device__ __forceinline__ float2 v2(c2 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ c2 c2v(float2 a) { return {a.x, a.y}; }
__device__ __forceinline__ float2 sw2(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float2 bc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// A complex coefficient split for packed multiplication.
struct CPk {
  float2 r, i;  // (m.x, m.x), (-m.y, m.y)
};
__device__ __forceinline__ CPk cpk(c2 m) { return {bc2(m.x), make_float2(-m.y, m.y)}; }
// m a, with as = sw2(a)
__device__ __forceinline__ float2 cmul_pk(const CPk& m, float2 a, float2 as) { return fma2(m.i, as, mul2(m.r, a)); }
__device__ __forceinline__ float2 cfma_pk(const CPk& m, float2 a, float2 as, float2 acc) {
  return fma2(m.i, as, fma2(m.r, a, acc));
}

struct M2Pk {
  CPk m00, m01, m10, m11;
};
__device__ __forceinline__ M2Pk m2pk(const M2& m) { return {cpk(m.m00), cpk(m.m01), cpk(m.m10), cpk(m.m11)}; }

// (a0, a1) -> (m00 a0 + m01 a1, m10 a0 + m11 a1), packed
__device__ __forceinline__ void apply2_pk(const M2Pk& m, c2& a0, c2& a1) {
  const float2 x0 = v2(a0), x1 = v2(a1), s0 = sw2(x0), s1 = sw2(x1);
  a0 = c2v(cfma_pk(m.m01, x1, s1, cmul_pk(m.m00, x0, s0)));
  a1 = c2v(cfma_pk(m.m11, x1, s1, cmul_pk(m.m10, x0, s0)));
}

// ------------------------------------------------------ register gate kernels

template <int M, int R>
__device__ __forceinline__ void reg_pair(c2 (&a)[1 << M], const M2& m) {
  const M2Pk mp = m2pk(m);
#pragma unroll
  for (int j = 0; j < (1 << M); j++) {
    if (j & (1 << R)) continue;
    apply2_pk(mp, a[j], a[j | (1 << R)]);
  }
}

template <int M, int R>
__device__ __forceinline__ void reg_swap(c2 (&a)[1 << M], int cbit_reg) {
  // swap across register bit R where the control (register bit cbit_reg, or
  // cbit_reg < 0: always) is 1
#pragma unroll
  for (int j = 0; j < (1 << M); j++) {
    if (j & (1 << R)) continue;
    if (cbit_reg >= 0 && !((j >> cbit_reg) & 1)) continue;
    const c2 t = a[j];
    a[j] = a[j | (1 << R)];
    a[j | (1 << R)] = t;
  }
}

template <int M>
__device__ __forceinline__ void reg_pair_any(c2 (&a)[1 << M], const M2& m, int r) {
  if (r == 0) reg_pair<M, 0>(a, m);
  else if (M > 1 && r == 1) reg_pair<M, (M > 1 ? 1 : 0)>(a, m);
  else if (M > 2 && r == 2) reg_pair<M, (M > 2 ? 2 : 0)>(a, m);
  else if (M > 3) reg_pair<M, (M > 3 ? 3 : 0)>(a, m);
}

template <int M>
__device__ __forceinline__ void reg_swap_any(c2 (&a)[1 << M], int r, int creg) {
  if (r == 0) reg_swap<M, 0>(a, creg);
  else if (M > 1 && r == 1) reg_swap<M, (M > 1 ? 1 : 0)>(a, creg);
  else if (M > 2 && r == 2) reg_swap<M, (M > 2 ? 2 : 0)>(a, creg);
  else if (M > 3) reg_swap<M, (M > 3 ? 3 : 0)>(a, creg);
}

// A compile-time integer carried as a type.
template <int V>
struct IC {
  static constexpr int value = V;
};

// Register-bit dispatch: call f with IC<R> for the
// runtime register bit r (R = -1 when r is not a register bit), so that the
// per-amplitude bit tests below are compile-time constants.
template <int M, typename F>
__device__ __forceinline__ void dispatch1(int r, F&& f) {
  switch (r) {
    case 0: f(IC<0>()); break;
    case 1: if constexpr (M > 1) f(IC<1>()); break;
    case 2: if constexpr (M > 2) f(IC<2>()); break;
    case 3: if constexpr (M > 3) f(IC<3>()); break;
    default: f(IC<-1>()); break;
  }
}

template <int M, typename F>
__device__ __forceinline__ void dispatch2(int r0, int r1, F&& f) {
  dispatch1<M>(r0, [&](auto A) { dispatch1<M>(r1, [&](auto B) { f(A, B); }); });
}

template <int R>
__device__ __forceinline__ constexpr int cbit(int j) {
  if constexpr (R < 0) return 0;
  else return (j >> R) & 1;
}

// Diagonal phase by the parity of register bits R0, R1 (either may be -1).
template <int M, int R0, int R1>
__device__ __forceinline__ void diag_par(c2 (&a)[1 << M], c2 d0, c2 d1) {
#pragma unroll
  for (int j = 0; j < (1 << M); j++) a[j] = cmul((cbit<R0>(j) ^ cbit<R1>(j)) ? d1 : d0, a[j]);
}

// Sign flip where register bits R0 and R1 are both 1 (CZ).
template <int M, int R0, int R1>
__device__ __forceinline__ void neg_and(c2 (&a)[1 << M]) {
#pragma unroll
  for (int j = 0; j < (1 << M); j++)
    if (cbit<R0>(j) & cbit<R1>(j)) a[j] = {-a[j].x, -a[j].y};
}

// Swap across register bit T where register bit C (or always, C = -1) is 1.
template <int M, int T, int C>
__device__ __forceinline__ void swap_ctrl(c2 (&a)[1 << M]) {
#pragma unroll
  for (int j = 0; j < (1 << M); j++) {
    if (j & (1 << T)) continue;
    if (C >= 0 && !cbit<C>(j)) continue;
    const c2 t = a[j];
    a[j] = a[j | (1 << T)];
    a[j | (1 << T)] = t;
  }
}

// Where an op's bit lives for the current group: register bit (0..M-1) or
// a bit value fixed for the group.
struct BitSrc {
  int reg;  // -1 if not a register bit
  int val;  // bit value when reg < 0
};

__device__ __forceinline__ BitSrc bsrc(int r, int l, int p, uint32_t gb, uint32_t base) {
  BitSrc s;
  s.reg = r;
  s.val = r >= 0 ? 0 : (l >= 0 ? (int)((gb >> l) & 1u) : (p >= 0 ? (int)((base >> p) & 1u) : 0));
  return s;
}

template <int M>
__device__ __forceinline__ int bit_of(const BitSrc& s, int j) {
  return s.reg >= 0 ? ((j >> s.reg) & 1) : s.val;
}

// Absorb op into the register group (dag: its adjoint).
template <int M>
__device__ __forceinline__ void reg_apply(c2 (&a)[1 << M], int kind, const OpMat& om,
                                          const BitSrc& b0, const BitSrc& b1, bool dag) {
  switch (kind) {
    case K_CNOT:  // target b1 is always a register bit
      if (b0.reg >= 0) {
        dispatch2<M>(b1.reg, b0.reg, [&](auto T, auto C) {
          constexpr int t = decltype(T)::value, c = decltype(C)::value;
          if constexpr (t >= 0 && c >= 0 && t != c) swap_ctrl<M, t, c>(a);
        });
      } else if (b0.val) {
        dispatch1<M>(b1.reg, [&](auto T) {
          constexpr int t = decltype(T)::value;
          if constexpr (t >= 0) swap_ctrl<M, t, -1>(a);
        });
      }
      return;
    case K_CZ:
      if (b0.reg >= 0 && b1.reg >= 0) {
        dispatch2<M>(b0.reg, b1.reg, [&](auto A, auto B) {
          constexpr int r0 = decltype(A)::value, r1 = decltype(B)::value;
          if constexpr (r0 >= 0 && r1 >= 0 && r0 != r1) neg_and<M, r0, r1>(a);
        });
      } else if (b0.reg >= 0 || b1.reg >= 0) {
        if (b0.reg >= 0 ? b1.val : b0.val)  // the fixed bit is 1: Z on the register bit
          dispatch1<M>(b0.reg >= 0 ? b0.reg : b1.reg, [&](auto A) {
            constexpr int r = decltype(A)::value;
            if constexpr (r >= 0) neg_and<M, r, r>(a);
          });
      } else if (b0.val & b1.val) {
#pragma unroll
        for (int j = 0; j < (1 << M); j++) a[j] = {-a[j].x, -a[j].y};
      }
      return;
    case K_RZZ: case K_RZ: case K_Z: {
      c2 d0 = om.m.m00, d1 = om.m.m11;
      if (dag) {
        d0.y = -d0.y;
        d1.y = -d1.y;
      }
      // parity of the bits; fixed bits flip the phase pair once per group
      const int fixed = (b0.reg < 0 ? b0.val : 0) ^ (kind == K_RZZ && b1.reg < 0 ? b1.val : 0);
      if (fixed) {
        const c2 t = d0;
        d0 = d1;
        d1 = t;
      }
      const int r0 = b0.reg, r1 = kind == K_RZZ ? b1.reg : -1;
      dispatch2<M>(r0, r1, [&](auto A, auto B) {
        diag_par<M, decltype(A)::value, decltype(B)::value>(a, d0, d1);
      });
      return;
    }
    default:
      reg_pair_any<M>(a, dag ? dagger(om.m) : om.m, b0.reg);
  }
}

// Adjoint of a diagonal rotation with its gradient share: s(x) = +-1 by the
// parity of register bits R0, R1; acc += s(x) Im(conj(lambda) psi), then
// psi, lambda times the conjugate phases.  Packed: Im(conj(l) p) = l.x p.y -
// l.y p.x is the difference of the halves of l . (p.y, p.x), which the phase
// multiplication of psi needs as well.
template <int M, int R0, int R1>
__device__ __forceinline__ void diag_par_adj(c2 (&p)[1 << M], c2 (&l)[1 << M], c2 d0, c2 d1, float& acc) {
  const CPk e0 = cpk(d0), e1 = cpk(d1);
  float2 g0 = make_float2(0.f, 0.f), g1 = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < (1 << M); j++) {
    const int bit = cbit<R0>(j) ^ cbit<R1>(j);
    const float2 x = v2(p[j]), y = v2(l[j]), xs = sw2(x);
    if (bit) g1 = fma2(y, xs, g1);
    else g0 = fma2(y, xs, g0);
    p[j] = c2v(cmul_pk(bit ? e1 : e0, x, xs));
    l[j] = c2v(cmul_pk(bit ? e1 : e0, y, sw2(y)));
  }
  acc += (g0.x - g0.y) - (g1.x - g1.y);
}

// One reverse-sweep step on the register group: un-compute psi, add the
// op's angle derivatives (this thread's share) into g, propagate lambda.
// Rules (psi_g = state after the gate, lambda_g its cotangent):
//   exp(-i t P/2) rotations: dF/dt = Im <lambda_g| P |psi_g>
//   U3: d/dtheta = 2 Re <lambda_g| dG/dtheta |psi_{g-1}>,
//       d/dphi = -2 Im(conj(lambda_g[1]) psi_g[1]),
//       d/dlambda = -2 Im(conj(lambda_{g-1}[1]) psi_{g-1}[1]).
// Rotation about X or Y by -t (the adjoint of RX(t) / RY(t)) applied to a
// pair, with c = cos t/2 and s = sin t/2 read from the gate tensor, packed
// over (re, im): RY(t)^dagger = [[c, s], [-s, c]] is real, so each output is
// c . a + (+-s) . b; RX(t)^dagger = [[c, i s], [i s, c]] multiplies the
// partner by i s, (-s, s) . (b.y, b.x).
__device__ __forceinline__ void ry_inv_pk(float2 C, float2 S, float2 NS, float2& a0, float2& a1) {
  const float2 b0 = fma2(C, a0, mul2(S, a1));
  const float2 b1 = fma2(C, a1, mul2(NS, a0));
  a0 = b0;
  a1 = b1;
}

__device__ __forceinline__ void rx_inv_pk(float2 C, float2 NSP, float2& a0, float2& a1) {
  const float2 b0 = fma2(NSP, sw2(a1), mul2(C, a0));
  const float2 b1 = fma2(NSP, sw2(a0), mul2(C, a1));
  a0 = b0;
  a1 = b1;
}

template <int M, int R>
__device__ __forceinline__ void reg_adj_1q(c2 (&p)[1 << M], c2 (&l)[1 << M], int kind, const OpMat& om,
                                           float* g) {
  if (kind == K_RY) {  // m00 = (c, 0), m01 = (-s, 0)
    const float c = om.m.m00.x, sn = -om.m.m01.x;
    const float2 C = bc2(c), S = bc2(sn), NS = bc2(-sn);
    // dF/dt = Im <lambda| Y |psi> = sum over pairs of l1.p0 - l0.p1 (real dots)
    float2 gp = make_float2(0.f, 0.f), gn = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < (1 << M); j++) {
      if (j & (1 << R)) continue;
      const int k = j | (1 << R);
      float2 p0 = v2(p[j]), p1 = v2(p[k]), l0 = v2(l[j]), l1 = v2(l[k]);
      gp = fma2(l1, p0, gp);
      gn = fma2(l0, p1, gn);
      ry_inv_pk(C, S, NS, p0, p1);
      ry_inv_pk(C, S, NS, l0, l1);
      p[j] = c2v(p0);
      p[k] = c2v(p1);
      l[j] = c2v(l0);
      l[k] = c2v(l1);
    }
    g[0] += (gp.x + gp.y) - (gn.x + gn.y);
    return;
  }
  if (kind == K_RX) {  // m00 = (c, 0), m01 = (0, -s)
    const float c = om.m.m00.x, sn = -om.m.m01.y;
    const float2 C = bc2(c), NSP = make_float2(-sn, sn);
    // dF/dt = Im <lambda| X |psi> = sum of Im(conj(l0) p1) + Im(conj(l1) p0)
    float2 gx = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < (1 << M); j++) {
      if (j & (1 << R)) continue;
      const int k = j | (1 << R);
      float2 p0 = v2(p[j]), p1 = v2(p[k]), l0 = v2(l[j]), l1 = v2(l[k]);
      gx = fma2(l0, sw2(p1), gx);
      gx = fma2(l1, sw2(p0), gx);
      rx_inv_pk(C, NSP, p0, p1);
      rx_inv_pk(C, NSP, l0, l1);
      p[j] = c2v(p0);
      p[k] = c2v(p1);
      l[j] = c2v(l0);
      l[k] = c2v(l1);
    }
    g[0] += gx.x - gx.y;
    return;
  }
  const M2Pk md = m2pk(dagger(om.m));
  M2Pk dd{};
  if (kind == K_U3) dd = m2pk(om.d);
#pragma unroll
  for (int j = 0; j < (1 << M); j++) {
    if (j & (1 << R)) continue;
    const int k = j | (1 << R);
    c2 p0 = p[j], p1 = p[k], l0 = l[j], l1 = l[k];
    if (kind == K_U3) g[1] += -2.f * (l1.x * p1.y - l1.y * p1.x);
    apply2_pk(md, p0, p1);
    if (kind == K_U3) {
      c2 d0 = p0, d1 = p1;
      apply2_pk(dd, d0, d1);
      const c2 z = cadd(cmulc(l0, d0), cmulc(l1, d1));
      g[0] += 2.f * z.x;
    }
    apply2_pk(md, l0, l1);
    if (kind == K_U3) g[2] += -2.f * (l1.x * p1.y - l1.y * p1.x);
    p[j] = p0;
    p[k] = p1;
    l[j] = l0;
    l[k] = l1;
  }
}

template <int M>
__device__ __forceinline__ void reg_adjoint(c2 (&p)[1 << M], c2 (&l)[1 << M], int kind,
                                            const OpMat& om, const BitSrc& b0, const BitSrc& b1,
                                            float* g) {
  switch (kind) {
    case K_CNOT: case K_CZ:
      reg_apply<M>(p, kind, om, b0, b1, true);
      reg_apply<M>(l, kind, om, b0, b1, true);
      return;
    case K_RZZ: case K_RZ: case K_Z: {
      c2 d0 = {om.m.m00.x, -om.m.m00.y}, d1 = {om.m.m11.x, -om.m.m11.y};
      const int fixed = (b0.reg < 0 ? b0.val : 0) ^ (kind == K_RZZ && b1.reg < 0 ? b1.val : 0);
      if (fixed) {  // a fixed 1 flips every amplitude's sign s(x) and phase
        const c2 t = d0;
        d0 = d1;
        d1 = t;
      }
      float acc = 0.f;
      dispatch2<M>(b0.reg, kind == K_RZZ ? b1.reg : -1, [&](auto A, auto B) {
        diag_par_adj<M, decltype(A)::value, decltype(B)::value>(p, l, d0, d1, acc);
      });
      g[0] += fixed ? -acc : acc;
      return;
    }
    default:
      if (b0.reg == 0) reg_adj_1q<M, 0>(p, l, kind, om, g);
      else if (M > 1 && b0.reg == 1) reg_adj_1q<M, (M > 1 ? 1 : 0)>(p, l, kind, om, g);
      else if (M > 2 && b0.reg == 2) reg_adj_1q<M, (M > 2 ? 2 : 0)>(p, l, kind, om, g);
      else if (M > 3) reg_adj_1q<M, (M > 3 ? 3 : 0)>(p, l, kind, om, g);
  }
}

// Tile-local base index of group grp: zeros inserted at the pass's bits.
template <int M>
__device__ __forceinline__ uint32_t group_base(const RegPass& rp, uint32_t grp) {
  uint32_t gb = grp;
#pragma unroll
  for (int i = 0; i < M; i++) gb = insert0(gb, rp.lb[i]);
  return gb;
}

template <int M>
__device__ __forceinline__ uint32_t group_off(const RegPass& rp, int j) {
  uint32_t o = 0;
#pragma unroll
  for (int i = 0; i < M; i++)
    if ((j >> i) & 1) o |= 1u << rp.lb[i];
  return o;
}

// Forward register pass over one group.  base: global index bits fixed for
// the tile (0 for a whole-state tile).
template <int M>
__device__ __forceinline__ void fwd_group(c2* st, const RegPass& rp, const DOp* dops,
                                          const OpMat* mats, uint32_t base, uint32_t grp) {
  constexpr int N = 1 << M;
  const uint32_t gb = group_base<M>(rp, grp);
  c2 a[N];
#pragma unroll
  for (int j = 0; j < N; j++) a[j] = st[swz(gb | group_off<M>(rp, j))];
  for (int o = rp.op_begin; o < rp.op_end; o++) {
    const DOp d = dops[o];
    const int kind = d.kind;
    if (kind == K_FUSED || kind == K_RX || kind == K_RY || kind == K_U3 || kind == K_H || kind == K_X ||
        kind == K_Y) {  // dense one-qubit: only the register bit is needed
      reg_pair_any<M>(a, mats[d.mat].m, d.r0);
      continue;
    }
    const BitSrc b0 = bsrc(d.r0, d.l0, d.p0, gb, base);
    const BitSrc b1 = (kind == K_RZ || kind == K_Z) ? BitSrc{-1, 0} : bsrc(d.r1, d.l1, d.p1, gb, base);
    reg_apply<M>(a, kind, mats[d.mat], b0, b1, false);
  }
#pragma unroll
  for (int j = 0; j < N; j++) st[swz(gb | group_off<M>(rp, j))] = a[j];
}

// Reverse register pass over one group; gradient shares are warp-reduced and
// added to gdst[slot] (PER_SLOT) or gdst[3 * d.mat + angle].
template <int M, bool PER_SLOT>
__device__ __forceinline__ void adj_group(c2* psi, c2* lam, const RegPass& rp, const DOp* dops,
                                          const OpMat* mats, uint32_t base, uint32_t grp, bool active,
                                          double* gdst) {
  constexpr int N = 1 << M;
  const uint32_t gb = group_base<M>(rp, grp);
  c2 p[N], l[N];
  if (active) {
#pragma unroll
    for (int j = 0; j < N; j++) {
      const uint32_t x = swz(gb | group_off<M>(rp, j));
      p[j] = psi[x];
      l[j] = lam[x];
    }
  }
  for (int o = rp.op_end - 1; o >= rp.op_begin; o--) {
    const DOp d = dops[o];
    float g[3] = {0.f, 0.f, 0.f};
    if (active) {
      const int kind = d.kind;
      const bool dense = kind == K_RX || kind == K_RY || kind == K_U3 || kind == K_H || kind == K_X || kind == K_Y;
      const BitSrc b0 = dense ? BitSrc{d.r0, 0} : bsrc(d.r0, d.l0, d.p0, gb, base);
      const BitSrc b1 = (dense || kind == K_RZ || kind == K_Z) ? BitSrc{-1, 0} : bsrc(d.r1, d.l1, d.p1, gb, base);
      reg_adjoint<M>(p, l, kind, mats[d.mat], b0, b1, g);
    }
#pragma unroll
    for (int j = 0; j < 3; j++) {
      if (j >= d.nang || d.slot[j] < 0) continue;
      const float v = warp_sum_f(g[j]);
      if ((threadIdx.x & 31) == 0)
        atomicAdd(PER_SLOT ? &gdst[d.slot[j]] : &gdst[3 * d.mat + j], (double)v);
    }
  }
  if (active) {
#pragma unroll
    for (int j = 0; j < N; j++) {
      const uint32_t x = swz(gb | group_off<M>(rp, j));
      psi[x] = p[j];
      lam[x] = l[j];
    }
  }
}

// Asynchronous 8-byte global -> shared copy (cp.async, completed in groups).
__device__ __forceinline__ void cp_async8(c2* dst_smem, const c2* src_gmem) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Wait until at most N of this thread's committed groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Warp-reduced gradient share v, added by lane 0 to entry `index` of its
// warp's own row (length `stride`) of partial sums: no atomics, each warp
// owns a row.
__device__ __forceinline__ void grad_share(float* gpart, int stride, int index, float v) {
  v = warp_sum_f(v);
  if ((threadIdx.x & 31) == 0) gpart[(threadIdx.x >> 5) * stride + index] += v;
}

// K (a power of two, <= 32) gradient shares reduced over the warp at once: a
// butterfly that halves the number of values at every exchange (lanes with
// the exchanged bit set keep the upper half), then a plain butterfly on the
// last value.  Afterwards lane l holds the warp total of value
// j = (l >> (5 - log2 K)) (the lane bits of the halving exchanges, high to
// low); lanes with the low 5 - log2 K bits clear add it to entry idx[j] of
// their warp's row (length stride) of partial sums.  K - 1 + (5 - log2 K)
// shuffles instead of 5 K.
template <int K>
__device__ __forceinline__ void grad_share_multi(float* gpart, int stride, const int* idx, float (&v)[K]) {
  static_assert(K >= 1 && K <= 32 && (K & (K - 1)) == 0, "K: a power of two up to 32");
  const int lane = threadIdx.x & 31;
  constexpr int LK = K == 1 ? 0 : K == 2 ? 1 : K == 4 ? 2 : K == 8 ? 3 : K == 16 ? 4 : 5;
#pragma unroll
  for (int st = 0; st < LK; st++) {
    const int o = 16 >> st;
    const int h = K >> (st + 1);  // values after this exchange
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < h; j++) {
      const float send = up ? v[j] : v[j + h];
      const float keep = up ? v[j + h] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (int o = 16 >> LK; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  constexpr int low = 5 - LK;
  if ((lane & ((1 << low) - 1)) == 0) gpart[(threadIdx.x >> 5) * stride + idx[lane >> low]] += v[0];
}

// Gate-tensor table of one row: recipe r multiplies the 2x2 tensors of ops
// rec_ops[rec_ptr[r] .. rec_ptr[r+1]) in order (a single op for unfused
// entries; two-qubit diagonal gates keep their phases).
__device__ __forceinline__ OpMat build_recipe(const SweepArgs& a, const SweepOp* ops, const int* rec_ptr,
                                              const int* rec_ops, int r, int64_t b, int k, int* bad) {
  const int e0 = rec_ptr[r], e1 = rec_ptr[r + 1];
  float ang[3] = {0.f, 0.f, 0.f};
  const int o0 = rec_ops[e0];
  const SweepOp op0 = ops[o0];
  row_angles(a, op0, o0, b, k, ang, bad);
  OpMat om = build_opmat(op0, ang);
  for (int e = e0 + 1; e < e1; e++) {  // fused one-qubit product: later gates on the left
    const int o = rec_ops[e];
    const SweepOp op = ops[o];
    row_angles(a, op, o, b, k, ang, bad);
    const M2 g = gate_1q(op.kind, ang);
    const M2 m = om.m;
    om.m.m00 = cfma(g.m01, m.m10, cmul(g.m00, m.m00));
    om.m.m01 = cfma(g.m01, m.m11, cmul(g.m00, m.m01));
    om.m.m10 = cfma(g.m11, m.m10, cmul(g.m10, m.m00));
    om.m.m11 = cfma(g.m11, m.m11, cmul(g.m10, m.m01));
  }
  return om;
}

}  // namespace tdq
