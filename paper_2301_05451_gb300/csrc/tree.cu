// Step (e) of Sec. 3.2 for an arbitrary pairwise path with sliced indices:
// the tree executor.
//
// Layout.  Every tensor of the path is stored in the order its consumer
// wants: the indices that survive the consumer first, then the consumer's
// contracted indices, sorted by id, as the lowest bits.  Step s = (A, B) is
// then exactly a batched "NT" product
//     C[m][n] = sum_k A[m][k] B[n][k],   m = A's outer bits, n = B's, k shared,
// with both operands contiguous in k, and the epilogue scatters C[m][n] into
// C's own consumer order.  The batch is (row, slice) pairs: slicing fixes the
// sliced indices' values in the leaves (Sec. 3.2.3, Eq. 8) and the slices'
// scalar results are summed in FP64 (K5).
//
// Kernels: every maximal subtree of small steps (all three tensors at most
// 2^11 entries) runs in one CTA per (subtree, row, slice) with its leaves
// (K0-tree, built from the angles), tensors and step table in shared memory,
// all subtrees in one launch; each remaining large step is one launch (K3:
// shared-memory tiled product for large m, n, k, else one thread per output
// entry).  The "plain" form runs every step as its own launch, one slice at a
// time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <utility>
#include <vector>

#include "cgemm_tc.cuh"
#include "graph_replay.h"
#include "network.h"
#include "sweep_common.cuh"
#include "tdq_internal.h"

namespace tdq {

namespace {

struct LeafDev {
  int8_t kind, gkind, conj, bit;
  int8_t rank;        // stored rank (sliced positions removed)
  int8_t rfull;       // rank before slicing
  int8_t flip;        // full position p complemented when bit p is set (anti-diagonal reduction)
  int8_t pos[4];      // full position i: stored bit position (>= 0) or -1 - (sliced index number)
  int32_t src[3];
  float fixed[3];
  int64_t off;        // arena offset (elements)
};

// One pairwise step C[h, m, n] = sum_k A[h][m][k] B[h][n][k]: h are the
// indices on A, B and C (hyperedges that continue past this step), k the
// summed ones; A and B are stored [h][m][k] / [h][n][k] (k fastest), C's bits
// wherever its own consumer wants them.
constexpr int kMaxHyperBits = 16;
struct StepDev {
  int64_t a_off, b_off, c_off;
  uint32_t pre;   // subtree steps: outputs of the earlier steps of the same level
  int8_t nm, nn, nk, rc, nh;
  int8_t cm[32];  // C bit position of m bit i (LSB first)
  int8_t cn[32];  // C bit position of n bit i
  int8_t ch[kMaxHyperBits];  // C bit position of h bit i
};

__device__ __forceinline__ float leaf_angle(const LeafDev& L, int j, const float* params, int64_t pstride,
                                            const float* inputs, int F, int64_t b, int* bad) {
  const int s = L.src[j];
  float v;
  if (s >= 0) v = params[b * pstride + s];
  else if (s == -1) v = L.fixed[j];
  else v = inputs[b * F + (-2 - s)];
  if (!isfinite(v)) *bad = 1;
  return v;
}

// Entry of a leaf tensor at full index bits v0[0..rfull) (v0[0] first index);
// complemented positions read the plain tensor at the other value.
__device__ c2 leaf_entry(const LeafDev& L, const int* v0, const float* ang) {
  int v[4];
#pragma unroll
  for (int p = 0; p < 4; p++) v[p] = v0[p] ^ ((L.flip >> p) & 1);
  c2 r = {0.f, 0.f};
  switch (L.kind) {
    case LEAF_KET0: r.x = v[0] == 0 ? 1.f : 0.f; break;
    case LEAF_BIT: r.x = v[0] == L.bit ? 1.f : 0.f; break;
    case LEAF_OBS_Z: r.x = v[0] == v[1] ? (v[0] ? -1.f : 1.f) : 0.f; break;
    case LEAF_HALF0: r.x = (v[1] == v[2] && v[2] == v[0]) ? 1.f : 0.f; break;
    case LEAF_DIAG: {  // diagonal of Z, RZ (one index), CZ, RZZ (two), or the Z observable
      if (L.gkind == K_RZ || L.gkind == K_RZZ) {
        const int odd = L.gkind == K_RZ ? v[0] : (v[0] ^ v[1]);
        float sn, cs;
        sincosf(0.5f * ang[0], &sn, &cs);
        r = {cs, odd ? sn : -sn};  // e^{-+i t/2}
      } else if (L.gkind == K_CZ) {
        r.x = (v[0] & v[1]) ? -1.f : 1.f;
      } else if (L.gkind == K_Y) {  // the phases Y[1 - i][i] of the input value: (i, -i)
        r.y = v[0] ? -1.f : 1.f;
      } else {  // Z gate or Z observable
        r.x = v[0] ? -1.f : 1.f;
      }
      break;
    }
    case LEAF_CTRL: r.x = v[1] == (v[2] ^ v[0]) ? 1.f : 0.f; break;  // (c, out, in)
    case LEAF_HALF1: {  // V_s[out][in], s = v[0]
      const int s = v[0], o = v[1], i = v[2];
      if (L.gkind == K_CNOT) r.x = (s ? (o != i) : (o == i)) ? 1.f : 0.f;
      else if (L.gkind == K_CZ) r.x = (o == i) ? ((s && o) ? -1.f : 1.f) : 0.f;
      else if (o == i) {  // RZZ: V_s = diag(e^{-i(-1)^(s xor o) t/2})
        float sn, cs;
        sincosf(0.5f * ang[0], &sn, &cs);
        r = {cs, (s ^ o) ? sn : -sn};
      }
      break;
    }
    default: {  // LEAF_GATE
      if (L.rfull == 2) {
        const M2 m = gate_1q(L.gkind, ang);
        const c2 e[4] = {m.m00, m.m01, m.m10, m.m11};
        r = e[v[0] * 2 + v[1]];
      } else {  // two-qubit: M[2 oa + ob][2 ia + ib]
        const int row = 2 * v[0] + v[1], col = 2 * v[2] + v[3];
        if (L.gkind == K_CNOT) r.x = (v[0] == v[2] && v[1] == (v[2] ^ v[3])) ? 1.f : 0.f;
        else if (L.gkind == K_CZ) r.x = row == col ? (row == 3 ? -1.f : 1.f) : 0.f;
        else if (row == col) {  // RZZ
          float sn, cs;
          sincosf(0.5f * ang[0], &sn, &cs);
          r = {cs, (v[0] ^ v[1]) ? sn : -sn};
        }
      }
    }
  }
  if (L.conj) r.y = -r.y;
  return r;
}

// d(entry)/d(angle j) of a leaf tensor (gate leaves only; 0 otherwise).
__device__ c2 leaf_entry_grad(const LeafDev& L, const int* v0, const float* ang, int j) {
  int v[4];
#pragma unroll
  for (int p = 0; p < 4; p++) v[p] = v0[p] ^ ((L.flip >> p) & 1);
  c2 r = {0.f, 0.f};
  float sn, cs;
  if (L.kind == LEAF_DIAG && (L.gkind == K_RZ || L.gkind == K_RZZ) && j == 0) {  // d/dt e^{-+i t/2}
    const int odd = L.gkind == K_RZ ? v[0] : (v[0] ^ v[1]);
    sincosf(0.5f * ang[0], &sn, &cs);
    r = {-0.5f * sn, odd ? 0.5f * cs : -0.5f * cs};
  } else if (L.kind == LEAF_HALF1 && L.gkind == K_RZZ && j == 0) {  // V_s[o][o] = e^{-i z t/2}, z = (-1)^(s xor o)
    if (v[1] == v[2]) {
      sincosf(0.5f * ang[0], &sn, &cs);
      const float z = (v[0] ^ v[1]) ? -1.f : 1.f;
      r = {-0.5f * z * z * sn, -0.5f * z * cs};  // d/dt (cos(z t/2) - i sin(z t/2))
    }
  } else if (L.kind == LEAF_GATE && L.rfull == 4 && L.gkind == K_RZZ && j == 0) {
    const int row = 2 * v[0] + v[1], col = 2 * v[2] + v[3];
    if (row == col) {
      sincosf(0.5f * ang[0], &sn, &cs);
      const float z = (v[0] ^ v[1]) ? -1.f : 1.f;
      r = {-0.5f * sn, -0.5f * z * cs};
    }
  } else if (L.kind == LEAF_GATE && L.rfull == 2) {
    const int o = v[0], i = v[1];
    sincosf(0.5f * ang[0], &sn, &cs);
    switch (L.gkind) {
      case K_RX:  // d/dt [[c, -is], [-is, c]]
        r = (o == i) ? c2{-0.5f * sn, 0.f} : c2{0.f, -0.5f * cs};
        break;
      case K_RY:  // d/dt [[c, -s], [s, c]]
        r = (o == i) ? c2{-0.5f * sn, 0.f} : c2{(o ? 0.5f : -0.5f) * cs, 0.f};
        break;
      case K_RZ:  // d/dt diag(e^{-it/2}, e^{it/2})
        if (o == i) r = o ? c2{-0.5f * sn, 0.5f * cs} : c2{-0.5f * sn, -0.5f * cs};
        break;
      case K_U3: {
        float sp, cp, sl, cl, spl, cpl;
        sincosf(ang[1], &sp, &cp);
        sincosf(ang[2], &sl, &cl);
        sincosf(ang[1] + ang[2], &spl, &cpl);
        if (j == 0) {  // theta
          const c2 e[4] = {{-0.5f * sn, 0.f}, {-0.5f * cl * cs, -0.5f * sl * cs}, {0.5f * cp * cs, 0.5f * sp * cs},
                           {-0.5f * cpl * sn, -0.5f * spl * sn}};
          r = e[o * 2 + i];
        } else if (j == 1) {  // phi: i * row 1
          if (o == 1) r = (i == 0) ? c2{-sp * sn, cp * sn} : c2{-spl * cs, cpl * cs};
        } else {  // lambda: i * column 1
          if (i == 1) r = (o == 0) ? c2{sl * sn, -cl * sn} : c2{-spl * cs, cpl * cs};
        }
        break;
      }
      default: break;
    }
  }
  if (L.conj) r.y = -r.y;
  return r;
}

// Fill every leaf of batch entry e = (row b, slice sigma) at arena + off.
__device__ void build_leaves(const LeafDev* leaves, int nleaves, c2* arena, const float* params,
                             int64_t pstride, const float* inputs, int F, int64_t b, uint32_t sigma,
                             int* bad, int tid, int nt) {
  for (int w = tid; w < nleaves * 16; w += nt) {
    const int li = w >> 4, e = w & 15;
    const LeafDev L = leaves[li];
    if (e >= (1 << L.rank)) continue;
    float ang[3];
#pragma unroll
    for (int j = 0; j < 3; j++) ang[j] = leaf_angle(L, j, params, pstride, inputs, F, b, bad);
    int v[4] = {0, 0, 0, 0};
    for (int p = 0; p < L.rfull; p++) {
      const int q = L.pos[p];
      v[p] = q >= 0 ? ((e >> q) & 1) : (int)((sigma >> (-1 - q)) & 1u);
    }
    arena[L.off + e] = leaf_entry(L, v, ang);
  }
}

// Start of every tree kernel: wait until the kernel before it in the stream
// has completed and its writes are visible (a launch with programmatic stream
// serialisation may be dispatched before then; without it this returns at
// once), then let the next kernel of the stream be dispatched early.  A kernel
// waits before its first memory access, so at most two grids overlap and no
// read or write can run ahead of the one before.
__device__ __forceinline__ void chain_start() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t scatter_bits(uint32_t x, const int8_t* pos, int n) {
  uint32_t r = 0;
  for (int i = 0; i < n; i++) r |= ((x >> i) & 1u) << pos[i];
  return r;
}

// One step for one batch entry, threads tid.. of nt: C[h][m][n] = sum_k A[h][m][k] B[h][n][k].
// Output o (in [h][m][n] order) of one step: the k-sum of A[h][m] . B[h][n]
// written at its place in C.
// One output o of a step: C[h][m][n] = sum_k A[h][m][k] B[h][n][k].  With
// kRot the sum starts at k = o mod K and wraps around: the lanes of a warp
// (consecutive outputs, operand rows K entries apart) then read different
// shared-memory banks instead of one (K >= 16 put every lane on one bank).
template <bool kRot = false>
__device__ __forceinline__ void step_out(const StepDev& s, c2* arena, uint32_t o) {
  const uint32_t K = 1u << s.nk, N = 1u << s.nn, MN = 1u << (s.nm + s.nn);
  const uint32_t h = o >> (s.nm + s.nn), m = (o & (MN - 1u)) >> s.nn, n = o & (N - 1u);
  const c2* a = arena + s.a_off + (size_t)((h << s.nm) | m) * K;
  const c2* bb = arena + s.b_off + (size_t)((h << s.nn) | n) * K;
  float re = 0.f, im = 0.f;
  for (uint32_t k0 = 0; k0 < K; k0++) {
    const uint32_t k = kRot ? ((k0 + o) & (K - 1u)) : k0;
    const c2 x = a[k], y = bb[k];
    re = fmaf(x.x, y.x, fmaf(-x.y, y.y, re));
    im = fmaf(x.x, y.y, fmaf(x.y, y.x, im));
  }
  arena[s.c_off + (scatter_bits(h, s.ch, s.nh) | scatter_bits(m, s.cm, s.nm) | scatter_bits(n, s.cn, s.nn))] = {re, im};
}

__device__ __forceinline__ uint32_t step_outputs(const StepDev& s) { return 1u << (s.nm + s.nn + s.nh); }

template <bool kRot = false>
__device__ void step_generic(const StepDev& s, c2* arena, int tid, int nt) {
  const uint32_t tot = step_outputs(s);
  for (uint32_t o = tid; o < tot; o += nt) step_out<kRot>(s, arena, o);
}

// Reverse of one step for one batch entry: from C's cotangent (at boff + the
// value offsets) the cotangents of both operands, which each step writes once
// (every tensor has one consumer):  Abar[m][k] = sum_n Cbar[m][n] B[n][k],
// Bbar[n][k] = sum_m Cbar[m][n] A[m][k]  (holomorphic: no conjugation).
__device__ void step_adjoint(const StepDev& s, c2* arena, int64_t boff, int tid, int nt) {
  const c2* A = arena + s.a_off;
  const c2* B = arena + s.b_off;
  const c2* Cb = arena + boff + s.c_off;
  c2* Ab = arena + boff + s.a_off;
  c2* Bb = arena + boff + s.b_off;
  const uint32_t K = 1u << s.nk, M = 1u << s.nm, N = 1u << s.nn, H = 1u << s.nh;
  for (uint32_t o = tid; o < H * M * K; o += nt) {
    const uint32_t h = o >> (s.nm + s.nk), m = (o >> s.nk) & (M - 1u), k = o & (K - 1u);
    const uint32_t cm = scatter_bits(h, s.ch, s.nh) | scatter_bits(m, s.cm, s.nm);
    const c2* Bh = B + (size_t)(h << s.nn) * K;
    float re = 0.f, im = 0.f;
    for (uint32_t n = 0; n < N; n++) {
      const c2 x = Cb[cm | scatter_bits(n, s.cn, s.nn)], y = Bh[(size_t)n * K + k];
      re = fmaf(x.x, y.x, fmaf(-x.y, y.y, re));
      im = fmaf(x.x, y.y, fmaf(x.y, y.x, im));
    }
    Ab[o] = {re, im};
  }
  for (uint32_t o = tid; o < H * N * K; o += nt) {
    const uint32_t h = o >> (s.nn + s.nk), n = (o >> s.nk) & (N - 1u), k = o & (K - 1u);
    const uint32_t cn = scatter_bits(h, s.ch, s.nh) | scatter_bits(n, s.cn, s.nn);
    const c2* Ah = A + (size_t)(h << s.nm) * K;
    float re = 0.f, im = 0.f;
    for (uint32_t m = 0; m < M; m++) {
      const c2 x = Cb[scatter_bits(m, s.cm, s.nm) | cn], y = Ah[(size_t)m * K + k];
      re = fmaf(x.x, y.x, fmaf(-x.y, y.y, re));
      im = fmaf(x.x, y.y, fmaf(x.y, y.x, im));
    }
    Bb[o] = {re, im};
  }
}

// dF/d(parameter) of one batch entry: Re sum_e Lbar[e] dL[e]/d(angle) over every
// gate leaf, added to gacc[b][column] (FP64).
__device__ void leaf_gradients(const LeafDev* leaves, int nleaves, const c2* arena, int64_t boff,
                               const float* params, int64_t pstride, const float* inputs, int F, int64_t b,
                               uint32_t sigma, double* gacc_row, int tid, int nt) {
  for (int w = tid; w < nleaves * 3; w += nt) {
    const int li = w / 3, j = w % 3;
    const LeafDev L = leaves[li];
    if (L.src[j] < 0 || (L.kind != LEAF_GATE && L.kind != LEAF_HALF1 && L.kind != LEAF_DIAG)) continue;
    float ang[3];
    int bad = 0;
    for (int q = 0; q < 3; q++) ang[q] = leaf_angle(L, q, params, pstride, inputs, F, b, &bad);
    double acc = 0.0;
    for (int e = 0; e < (1 << L.rank); e++) {
      int v[4] = {0, 0, 0, 0};
      for (int p = 0; p < L.rfull; p++) {
        const int q = L.pos[p];
        v[p] = q >= 0 ? ((e >> q) & 1) : (int)((sigma >> (-1 - q)) & 1u);
      }
      const c2 d = leaf_entry_grad(L, v, ang, j);
      const c2 lb = arena[boff + L.off + e];
      acc += (double)(lb.x * d.x - lb.y * d.y);
    }
    atomicAdd(&gacc_row[L.src[j]], acc);
  }
}

struct TreeArgs {
  const LeafDev* leaves;
  int nleaves;
  const StepDev* steps;
  int nsteps;
  int64_t arena_elems;
  int64_t root_off;
  const float* params;
  int64_t pstride;
  const float* inputs;
  int F;
  int B;            // rows
  int chunk;        // slices per batch of this launch
  uint32_t slice0;  // first slice of the batch
  c2* work;         // [B * chunk][arena] (plain mode)
  c2* roots;        // [B * chunk]
  int* status;
  // reverse tree (gradients)
  int64_t boff;        // cotangent region offset in the arena
  const double* gw;    // [B] weights of the outputs, NULL = 1
  double coeff;        // term coefficient
  double* gacc;        // [B][P] FP64 gradient sums
  int P;
  const LeafDev* gleaves;  // leaves with workspace offsets (plain reverse)
};

// A subtree of small steps: its leaves and steps run in one CTA with every
// tensor (and the step descriptors) in shared memory; its root goes to the
// global workspace (or, for the network's root, to roots[]).
struct SubDev {
  int leaf_begin, leaf_end;
  int step_begin, step_end;
  int lev_begin, nlev;  // level bounds (relative step indices) at slev[lev_begin .. lev_begin + nlev]
  int smem_elems;       // shared arena (complex64 entries)
  int root_local;       // offset of the root in the shared arena
  int root_size;        // entries
  int64_t root_global;  // offset in the global arena, or -1: the network's root
};

__global__ void __launch_bounds__(512) k_tree_subtrees(TreeArgs a, const SubDev* subs, const LeafDev* sleaves,
                                                       const StepDev* ssteps, const int* slev) {
  chain_start();
  extern __shared__ __align__(16) unsigned char raw[];
  const SubDev sd = subs[blockIdx.x];
  c2* arena = reinterpret_cast<c2*>(raw);
  StepDev* st = reinterpret_cast<StepDev*>(arena + sd.smem_elems);
  const int e = blockIdx.y;
  const int64_t b = e / a.chunk;
  const uint32_t sigma = a.slice0 + (uint32_t)(e % a.chunk);
  const int ns = sd.step_end - sd.step_begin;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) st[i] = ssteps[sd.step_begin + i];
  int bad = 0;
  build_leaves(sleaves + sd.leaf_begin, sd.leaf_end - sd.leaf_begin, arena, a.params, a.pstride, a.inputs, a.F, b,
               sigma, &bad, threadIdx.x, blockDim.x);
  if (bad) atomicOr(a.status, 1 << TDQ_ERR_NONFINITE);
  __syncthreads();
  // level by level: the steps of a level are independent (their operands
  // come from earlier levels, and the arena keeps them apart), so the level's
  // outputs are shared out over the CTA as one range, one barrier per level
  for (int l = 0; l < sd.nlev; l++) {
    const int s0 = slev[sd.lev_begin + l], s1 = slev[sd.lev_begin + l + 1];
    const uint32_t total = st[s1 - 1].pre + step_outputs(st[s1 - 1]);
    int i = s0;
    for (uint32_t o = threadIdx.x; o < total; o += blockDim.x) {
      while (o >= st[i].pre + step_outputs(st[i])) i++;
      step_out<true>(st[i], arena, o - st[i].pre);
    }
    __syncthreads();
  }
  if (sd.root_global < 0) {
    if (threadIdx.x == 0) a.roots[e] = arena[sd.root_local];
  } else {
    c2* dst = a.work + (size_t)e * a.arena_elems + sd.root_global;
    for (int i = threadIdx.x; i < sd.root_size; i += blockDim.x) dst[i] = arena[sd.root_local + i];
  }
}

// Value and gradient of a whole small network in one CTA: leaves, forward
// steps, the root, then the reverse tree and the leaf gradients, every
// tensor and cotangent in shared memory (values at value offsets, cotangents
// at boff + value offsets).
__global__ void __launch_bounds__(128) k_tree_fused_adj(TreeArgs a, const LeafDev* leaves, int nleaves,
                                                        const StepDev* steps, int nsteps, int root_local,
                                                        int smem_elems) {
  chain_start();
  extern __shared__ __align__(16) unsigned char raw[];
  c2* arena = reinterpret_cast<c2*>(raw);
  StepDev* st = reinterpret_cast<StepDev*>(arena + smem_elems);
  const int e = blockIdx.x;
  const int64_t b = e / a.chunk;
  const uint32_t sigma = a.slice0 + (uint32_t)(e % a.chunk);
  for (int i = threadIdx.x; i < nsteps; i += blockDim.x) st[i] = steps[i];
  int bad = 0;
  build_leaves(leaves, nleaves, arena, a.params, a.pstride, a.inputs, a.F, b, sigma, &bad, threadIdx.x, blockDim.x);
  if (bad) atomicOr(a.status, 1 << TDQ_ERR_NONFINITE);
  __syncthreads();
  for (int i = 0; i < nsteps; i++) {
    step_generic<true>(st[i], arena, threadIdx.x, blockDim.x);  // shared-memory arena
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.roots[e] = arena[root_local];
    arena[a.boff + root_local] = {(float)((a.gw ? a.gw[b] : 1.0) * a.coeff), 0.f};
  }
  __syncthreads();
  for (int i = nsteps - 1; i >= 0; i--) {
    step_adjoint(st[i], arena, a.boff, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  leaf_gradients(leaves, nleaves, arena, a.boff, a.params, a.pstride, a.inputs, a.F, b, sigma, a.gacc + b * a.P,
                 threadIdx.x, blockDim.x);
}

// Plain reverse tree: the root's cotangent, one launch per step, leaf gradients.
__global__ void k_tree_root_bar(TreeArgs a) {
  chain_start();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.B * a.chunk) return;
  const int64_t b = e / a.chunk;
  a.work[(size_t)e * a.arena_elems + a.boff + a.root_off] = {(float)((a.gw ? a.gw[b] : 1.0) * a.coeff), 0.f};
}

__global__ void __launch_bounds__(256) k_tree_step_adj(TreeArgs a, int s) {
  chain_start();
  step_adjoint(a.steps[s], a.work + (size_t)blockIdx.y * a.arena_elems, a.boff, blockIdx.x * blockDim.x + threadIdx.x,
               gridDim.x * blockDim.x);
}

__global__ void k_tree_leaf_grads(TreeArgs a) {
  chain_start();
  const int e = blockIdx.y;
  const int64_t b = e / a.chunk;
  const uint32_t sigma = a.slice0 + (uint32_t)(e % a.chunk);
  leaf_gradients(a.gleaves, a.nleaves, a.work + (size_t)e * a.arena_elems, a.boff, a.params, a.pstride, a.inputs,
                 a.F, b, sigma, a.gacc + b * a.P, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void k_tree_grads_out(const double* gacc, int n, float* grads) {
  chain_start();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) grads[i] = (float)gacc[i];
}

// Large k, few outputs: one warp per output entry, lanes striding over k
// (both operands are k-contiguous), shuffle reduction.
__global__ void __launch_bounds__(256) k_tree_step_warp(TreeArgs a, int s) {
  chain_start();
  const StepDev st = a.steps[s];
  c2* base = a.work + (size_t)blockIdx.y * a.arena_elems;
  const c2* A = base + st.a_off;
  const c2* B = base + st.b_off;
  c2* C = base + st.c_off;
  const uint32_t K = 1u << st.nk, N = 1u << st.nn, MN = 1u << (st.nm + st.nn), tot = MN << st.nh;
  const int lane = threadIdx.x & 31;
  const uint32_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t o = w0; o < tot; o += nw) {
    const uint32_t h = o >> (st.nm + st.nn), m = (o & (MN - 1u)) >> st.nn, n = o & (N - 1u);
    const c2* x = A + (size_t)((h << st.nm) | m) * K;
    const c2* y = B + (size_t)((h << st.nn) | n) * K;
    float re = 0.f, im = 0.f;
#pragma unroll 8  // several loads in flight per lane
    for (uint32_t k = lane; k < K; k += 32) {
      const c2 u = x[k], v = y[k];
      re = fmaf(u.x, v.x, fmaf(-u.y, v.y, re));
      im = fmaf(u.x, v.y, fmaf(u.y, v.x, im));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, d);
      im += __shfl_xor_sync(0xffffffffu, im, d);
    }
    if (lane == 0) C[scatter_bits(h, st.ch, st.nh) | scatter_bits(m, st.cm, st.nm) | scatter_bits(n, st.cn, st.nn)] = {re, im};
  }
}

// Few outputs, long k: split k.  Block (c, e) sums k in [c KC, (c + 1) KC)
// for every output of batch entry e from operand chunks staged in shared
// memory, and adds its partial sums to C (zeroed before the launch) with FP32
// atomics.  With fewer than 256 outputs, 256 / outputs consecutive lanes share
// one (the kind rule sends 1..4096 outputs here); lanes of one output reduce
// within their warp, and each warp's sum is added separately.
constexpr int kSplitSmemC2 = 6144;  // staged complex operands per block (48 KiB)
__global__ void __launch_bounds__(256) k_tree_step_splitk(TreeArgs a, int s, int kc_log2) {
  chain_start();
  extern __shared__ __align__(16) unsigned char sk_raw[];
  c2* As = reinterpret_cast<c2*>(sk_raw);
  const StepDev st = a.steps[s];
  c2* base = a.work + (size_t)blockIdx.y * a.arena_elems;
  const c2* A = base + st.a_off;
  const c2* B = base + st.b_off;
  c2* C = base + st.c_off;
  const uint32_t K = 1u << st.nk, N = 1u << st.nn, KC = 1u << kc_log2;
  const uint32_t HM = 1u << (st.nh + st.nm), HN = 1u << (st.nh + st.nn), MN = 1u << (st.nm + st.nn);
  const uint32_t tot = MN << st.nh, k0 = blockIdx.x * KC;
  c2* Bs = As + HM * KC;
  // chunk rows: As[hm][kk] = A[hm][k0 + kk], Bs[hn][kk] = B[hn][k0 + kk] (coalesced along k)
  for (uint32_t i = threadIdx.x; i < HM * KC; i += blockDim.x) As[i] = A[(size_t)(i >> kc_log2) * K + k0 + (i & (KC - 1))];
  for (uint32_t i = threadIdx.x; i < HN * KC; i += blockDim.x) Bs[i] = B[(size_t)(i >> kc_log2) * K + k0 + (i & (KC - 1))];
  __syncthreads();
  // lanes per output: 256 / tot (1..16 for tot >= 16), consecutive lanes of a warp
  const uint32_t lpo = tot >= 256 ? 1u : 256u / tot;
  const uint32_t lane_o = threadIdx.x % lpo;
  for (uint32_t o = threadIdx.x / lpo; o < tot; o += blockDim.x / lpo) {
    const uint32_t h = o >> (st.nm + st.nn), m = (o & (MN - 1u)) >> st.nn, n = o & (N - 1u);
    const c2* x = As + ((h << st.nm) | m) * KC;
    const c2* y = Bs + ((h << st.nn) | n) * KC;
    float re = 0.f, im = 0.f;
    for (uint32_t kk = lane_o; kk < KC; kk += lpo) {
      // rotate the start so that lanes reading different rows hit different banks
      const uint32_t q = (kk + (n & 31u)) & (KC - 1u);
      const c2 u = x[q], v = y[q];
      re = fmaf(u.x, v.x, fmaf(-u.y, v.y, re));
      im = fmaf(u.x, v.y, fmaf(u.y, v.x, im));
    }
    const uint32_t red = lpo < 32u ? lpo : 32u;  // lanes of this output within one warp
    for (uint32_t d = red >> 1; d > 0; d >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, d);
      im += __shfl_xor_sync(0xffffffffu, im, d);
    }
    if (lane_o % red == 0) {
      float* c = reinterpret_cast<float*>(
          &C[scatter_bits(h, st.ch, st.nh) | scatter_bits(m, st.cm, st.nm) | scatter_bits(n, st.cn, st.nn)]);
      atomicAdd(c, re);
      atomicAdd(c + 1, im);
    }
  }
}

// One step for every batch entry: grid.y = batch entries.
__global__ void __launch_bounds__(256) k_tree_step(TreeArgs a, int s) {
  chain_start();
  const StepDev st = a.steps[s];
  step_generic(st, a.work + (size_t)blockIdx.y * a.arena_elems, blockIdx.x * blockDim.x + threadIdx.x,
               gridDim.x * blockDim.x);
}

// Large steps: 64x64 output tiles of C[m][n] = sum_k A[m][k] B[n][k] through
// shared memory (K3 in SIMT FP32), scattered epilogue.
constexpr int TM = 64, TN = 64, TK = 16;
__global__ void __launch_bounds__(256) k_tree_gemm(TreeArgs a, int s) {
  chain_start();
  __shared__ c2 As[TK][TM + 1];
  __shared__ c2 Bs[TK][TN + 1];
  const StepDev st = a.steps[s];
  const uint32_t M = 1u << st.nm, N = 1u << st.nn, K = 1u << st.nk;
  const uint32_t h = blockIdx.z & ((1u << st.nh) - 1u);  // grid.z = batch entries x 2^nh
  c2* base = a.work + (size_t)(blockIdx.z >> st.nh) * a.arena_elems;
  const c2* A = base + st.a_off + (size_t)h * M * K;
  const c2* Bm = base + st.b_off + (size_t)h * N * K;
  c2* C = base + st.c_off + scatter_bits(h, st.ch, st.nh);
  const uint32_t m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 4 x 4 outputs each
  float cr[4][4], ci[4][4];
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) cr[i][j] = ci[i][j] = 0.f;
  for (uint32_t k0 = 0; k0 < K; k0 += TK) {
    for (int t = threadIdx.x; t < TK * TM; t += 256) {
      const int kk = t % TK, mm = t / TK;
      const uint32_t m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? A[(size_t)m * K + k] : c2{0.f, 0.f};
      const uint32_t n = n0 + mm;
      Bs[kk][mm] = (n < N && k < K) ? Bm[(size_t)n * K + k] : c2{0.f, 0.f};
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; kk++) {
      c2 av[4], bv[4];
      for (int i = 0; i < 4; i++) av[i] = As[kk][ty * 4 + i];
      for (int j = 0; j < 4; j++) bv[j] = Bs[kk][tx * 4 + j];
      for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
          cr[i][j] = fmaf(av[i].x, bv[j].x, fmaf(-av[i].y, bv[j].y, cr[i][j]));
          ci[i][j] = fmaf(av[i].x, bv[j].y, fmaf(av[i].y, bv[j].x, ci[i][j]));
        }
    }
    __syncthreads();
  }
  for (int i = 0; i < 4; i++) {
    const uint32_t m = m0 + ty * 4 + i;
    if (m >= M) continue;
    const uint32_t cmb = scatter_bits(m, st.cm, st.nm);
    for (int j = 0; j < 4; j++) {
      const uint32_t n = n0 + tx * 4 + j;
      if (n >= N) continue;
      C[cmb | scatter_bits(n, st.cn, st.nn)] = {cr[i][j], ci[i][j]};
    }
  }
}

__global__ void k_tree_roots(TreeArgs a) {
  chain_start();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.B * a.chunk) return;
  a.roots[e] = a.work[(size_t)e * a.arena_elems + a.root_off];
}

// K5: FP64 sum of each row's slice results, in slice order (deterministic).
__global__ void k_slice_sum(const c2* roots, int B, int chunk, double* acc, int first) {
  chain_start();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double re = first ? 0.0 : acc[2 * b], im = first ? 0.0 : acc[2 * b + 1];
  for (int s = 0; s < chunk; s++) {
    const c2 v = roots[(size_t)b * chunk + s];
    re += (double)v.x;
    im += (double)v.y;
  }
  acc[2 * b] = re;
  acc[2 * b + 1] = im;
}

__global__ void k_tree_out(const double* acc, int B, int output, double coeff, double* values) {
  chain_start();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  if (output == TDQ_OUT_EXPVAL) values[b] = coeff * acc[2 * b];
  else {
    values[2 * b] = acc[2 * b];
    values[2 * b + 1] = acc[2 * b + 1];
  }
}

}  // namespace

// Launch with programmatic stream serialisation: the kernel may be
// dispatched while the kernel before it in the stream is finishing (it
// waits in chain_start).  Errors are also left for cudaGetLastError, as a
// <<< >>> launch leaves them.
template <typename... KArgs, typename... Args>
static cudaError_t launch_chained(void (*k)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t st,
                                  Args&&... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

struct TreeExec final : tdq_exec {
  int dev = 0, B = 0, P = 0, F = 0, output = 0, plain = 0;
  double coeff = 1.0;
  int n_sliced = 0;
  int64_t n_slices = 1;
  int64_t slice_lo = 0, slice_hi = -1;  // slices contracted by execute (hi < 0: all)
  int chunk = 1;
  int64_t arena = 0, root_off = -1;  // global arena; root_off < 0: a subtree writes the root
  std::vector<StepDev> steps_h;      // global (large) steps
  std::vector<int> step_kind;        // 0 thread per entry, 1 SIMT tiled, 2 tensor core (A as X),
                                     // 3 tensor core (B as X), 4 warp per entry (large k)
  LeafDev* d_sleaves = nullptr;      // leaves of the subtrees (shared-arena offsets)
  StepDev* d_ssteps = nullptr;       // steps of the subtrees (shared-arena offsets)
  SubDev* d_subs = nullptr;
  int* d_slev = nullptr;             // level bounds of the subtrees' steps
  int nsub = 0;
  size_t sub_smem = 0;
  int sm_count = 0;                  // SMs of the device (the subtree launch's CTA size follows its grid)
  int nleaves_g = 0;
  StepDev* d_steps = nullptr;
  int nsteps = 0;
  c2* d_work = nullptr;
  c2* d_roots = nullptr;
  double* d_acc = nullptr;
  int* d_status = nullptr;
  int last_launches = 0;
  cudaStream_t last_stream = nullptr;
  double flops_row = 0, bytes_row = 0;
  std::vector<cudaEvent_t> ev;  // K9: a (start, end) pair per launch unit of the first slice batch
  // reverse tree: 0 none, 1 fused (one CTA per row and slice), 2 plain (a launch per step)
  int adj = 0;
  int64_t boff = 0;
  LeafDev* d_fleaves = nullptr;  // fused reverse: leaves / steps with shared-arena offsets
  StepDev* d_fsteps = nullptr;
  int nfleaves = 0, nfsteps = 0, froot = 0, fsmem_elems = 0;
  size_t fsmem = 0;
  LeafDev* d_gleaves = nullptr;  // plain reverse: leaves with workspace offsets
  double* d_gacc = nullptr;
  // recomputing reverse (adj 3): the step descriptors of every region, its
  // range [reg_begin[r], reg_begin[r + 1]) in processing order (the root's
  // region first); the last step of a region makes its root (a checkpoint)
  std::vector<StepDev> rsteps_h;
  std::vector<int> rstep_kind, reg_begin;
  StepDev* d_rsteps = nullptr;
  // concurrent large steps: step s runs on stream step_stream[s] (0 = the
  // caller's stream, k > 0 = side[k - 1]) after the steps in step_waits[s]
  // on other streams; step_ev[s] is recorded after s when another stream waits for it
  std::vector<int> step_stream;
  std::vector<std::vector<int>> step_waits;
  std::vector<cudaEvent_t> step_ev;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> join_ev;
  cudaEvent_t fork_ev = nullptr;
  // the whole forward execution replayed as a CUDA graph while a call's
  // pointers, stride and stream repeat (values-only, not plain, not timed)
  bool use_graph = false;
  GraphReplay graph;

  ~TreeExec() override {
    for (cudaEvent_t x : ev) cudaEventDestroy(x);
    for (cudaEvent_t x : step_ev)
      if (x) cudaEventDestroy(x);
    for (cudaEvent_t x : join_ev) cudaEventDestroy(x);
    if (fork_ev) cudaEventDestroy(fork_ev);
    for (cudaStream_t x : side) cudaStreamDestroy(x);
    cudaFree(d_fleaves);
    cudaFree(d_fsteps);
    cudaFree(d_gleaves);
    cudaFree(d_rsteps);
    cudaFree(d_gacc);
    cudaFree(d_sleaves);
    cudaFree(d_ssteps);
    cudaFree(d_subs);
    cudaFree(d_slev);
    cudaFree(d_steps);
    cudaFree(d_work);
    cudaFree(d_roots);
    cudaFree(d_acc);
    cudaFree(d_status);
  }

  // One large step for nb batch entries on stream st (descriptors: host H,
  // device D == a.steps, kinds K; default: the forward steps).
  tdq_status launch_step(const TreeArgs& a, int s, int nb, cudaStream_t st) {
    return launch_step_of(a, s, nb, st, steps_h, d_steps, step_kind);
  }
  tdq_status launch_step_of(const TreeArgs& a, int s, int nb, cudaStream_t st, const std::vector<StepDev>& H,
                            const StepDev* D, const std::vector<int>& K) {
    const StepDev& sd = H[s];
    const std::vector<int>& step_kind = K;
    if (step_kind[s] == 2 || step_kind[s] == 3) {
      const bool ax = step_kind[s] == 2;
      const StepDev* dd = D + s;
      CgemmOut map{ax ? dd->cm : dd->cn, ax ? dd->cn : dd->cm, ax ? sd.nm : sd.nn, ax ? sd.nn : sd.nm, 0};
      const float2* w = reinterpret_cast<const float2*>(d_work);
      const char* where = "";
      cudaError_t ce = cudaSuccess;
      // one product per value of the hyperedge bits: operand blocks at h M K and
      // h N K, the result's h bits a constant offset
      for (uint32_t h = 0; h < (1u << sd.nh) && ce == cudaSuccess; h++) {
        uint32_t ch = 0;
        for (int i = 0; i < sd.nh; i++) ch |= ((h >> i) & 1u) << sd.ch[i];
        const int64_t ha = (int64_t)h << (sd.nm + sd.nk), hb = (int64_t)h << (sd.nn + sd.nk);
        ce = cgemm_tc_launch(w + (ax ? sd.a_off + ha : sd.b_off + hb), arena, w + (ax ? sd.b_off + hb : sd.a_off + ha),
                             arena, reinterpret_cast<float2*>(d_work) + sd.c_off + ch, arena,
                             1 << (ax ? sd.nm : sd.nn), 1 << (ax ? sd.nn : sd.nm), 1 << sd.nk, nb, map, d_status, st,
                             &where);
      }
      if (ce != cudaSuccess)
        return fail(TDQ_ERR_CUDA, std::string("tensor-core step (") + where + ", I " +
                                  std::to_string(1 << (ax ? sd.nm : sd.nn)) + " J " +
                                  std::to_string(1 << (ax ? sd.nn : sd.nm)) + " K " + std::to_string(1 << sd.nk) +
                                  " batch " + std::to_string(nb) + "): " + cudaGetErrorString(ce));
    } else if (step_kind[s] == 1 && ((int64_t)nb << sd.nh) <= 65535) {
      const dim3 g((unsigned)(((1u << sd.nn) + TN - 1) / TN), (unsigned)(((1u << sd.nm) + TM - 1) / TM),
                   (unsigned)nb << sd.nh);
      (void)launch_chained(k_tree_gemm, dim3(g), dim3(256), 0, st, a, s);
    } else if (step_kind[s] == 5) {
      // chunk of k: the largest power of two that keeps both operand chunks in 48 KiB
      const int mn = ((1 << sd.nm) + (1 << sd.nn)) << sd.nh;
      int kcl = 0;
      while (kcl < sd.nk && ((int64_t)mn << (kcl + 1)) <= kSplitSmemC2) kcl++;
      const size_t csize = sizeof(c2) << (sd.nh + sd.nm + sd.nn);
      if (cudaMemset2DAsync(reinterpret_cast<c2*>(d_work) + sd.c_off, (size_t)arena * sizeof(c2), 0, csize, nb, st) !=
          cudaSuccess)
        return fail(TDQ_ERR_CUDA, "step " + std::to_string(s) + ": clearing the split-k output");
      (void)launch_chained(k_tree_step_splitk, dim3(1u << (sd.nk - kcl), nb), dim3(256),
                           sizeof(c2) * ((size_t)mn << kcl), st, a, s, kcl);
    } else if (step_kind[s] == 4) {
      const int64_t tot = (int64_t)1 << (sd.nh + sd.nm + sd.nn);
      const unsigned blocks = (unsigned)std::min<int64_t>((tot * 32 + 255) / 256, 8192);
      (void)launch_chained(k_tree_step_warp, dim3(blocks, nb), dim3(256), 0, st, a, s);
    } else {  // a thread per output (also SIMT-tile steps whose batch x 2^h exceeds grid.z)
      const int64_t tot = (int64_t)1 << (sd.nh + sd.nm + sd.nn);
      const unsigned blocks = (unsigned)std::min<int64_t>((tot + 255) / 256, 4096);
      (void)launch_chained(k_tree_step, dim3(blocks, nb), dim3(256), 0, st, a, s);
    }
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess)
      return fail(TDQ_ERR_CUDA, "step " + std::to_string(s) + " (kind " + std::to_string(step_kind[s]) +
                                ", m " + std::to_string(sd.nm) + " n " + std::to_string(sd.nn) + " k " +
                                std::to_string(sd.nk) + ", batch " + std::to_string(nb) + "): " +
                                cudaGetErrorString(le));
    return TDQ_OK;
  }

  tdq_status execute(const float* params, int64_t pstride, const float* inputs, double* values,
                     const double* gw, float* grads, void* stream) override {
    if (!values) return fail(TDQ_ERR_ARG, "tdq_execute: values is NULL");
    if (P > 0 && !params) return fail(TDQ_ERR_ARG, "tdq_execute: params is NULL");
    if (F > 0 && !inputs) return fail(TDQ_ERR_ARG, "tdq_execute: inputs is NULL");
    if (pstride != 0 && pstride < P) return fail(TDQ_ERR_ARG, "tdq_execute: params_stride < P");
    if (!adj && (grads || gw)) return fail(TDQ_ERR_ARG, "tdq_execute: gradients given to a values-only exec");
    if (adj && !grads) return fail(TDQ_ERR_ARG, "tdq_execute: grads is NULL");
    TDQ_CUDA_TRY(cudaSetDevice(dev));
    cudaStream_t st = (cudaStream_t)stream;
    last_stream = st;
    if (!use_graph) return enqueue(params, pstride, inputs, values, gw, grads, st);
    const void* key[6] = {params, inputs, values, gw, grads, stream};
    return graph.run(key, pstride, st, &last_launches,
                     [&](cudaStream_t s2) { return enqueue(params, pstride, inputs, values, gw, grads, s2); });
  }

  // Enqueue one execution on stream st (the caller's, or the capture stream).
  tdq_status enqueue(const float* params, int64_t pstride, const float* inputs, double* values, const double* gw,
                     float* grads, cudaStream_t st) {
    last_launches = 0;
    TreeArgs a{};
    a.steps = d_steps;
    a.nsteps = nsteps;
    a.arena_elems = arena;
    a.root_off = root_off;
    a.params = params;
    a.pstride = pstride;
    a.inputs = inputs;
    a.F = F;
    a.B = B;
    a.work = d_work;
    a.roots = d_roots;
    a.status = d_status;
    a.boff = boff;
    a.gw = gw;
    a.coeff = coeff;
    a.gacc = d_gacc;
    a.P = P;
    a.gleaves = d_gleaves;
    if (adj) TDQ_CUDA_TRY(cudaMemsetAsync(d_gacc, 0, sizeof(double) * (size_t)B * std::max(1, P), st));
    const int64_t s_lo = slice_lo, s_hi = slice_hi < 0 ? n_slices : slice_hi;
    if (s_lo >= s_hi)  // an empty slice range: the partial sums are zero
      TDQ_CUDA_TRY(cudaMemsetAsync(d_acc, 0, sizeof(double) * 2 * (size_t)B, st));
    for (int64_t s0 = s_lo; s0 < s_hi; s0 += chunk) {
      a.chunk = (int)std::min<int64_t>(chunk, s_hi - s0);
      a.slice0 = (uint32_t)s0;
      const int nb = B * a.chunk;
      if (adj == 1) {  // value and gradient of the whole network per CTA
        (void)launch_chained(k_tree_fused_adj, dim3(nb), dim3(128), fsmem, st, a, d_fleaves, nfleaves, d_fsteps,
                             nfsteps, froot, fsmem_elems);
        last_launches++;
        TDQ_CUDA_TRY(cudaGetLastError());
        (void)launch_chained(k_slice_sum, dim3((B + 127) / 128), dim3(128), 0, st, d_roots, B, a.chunk, d_acc,
                             s0 == s_lo);
        last_launches++;
        continue;
      }
      const bool rec = !ev.empty() && s0 == s_lo;
      if (rec) cudaEventRecord(ev[0], st);
      // a level's outputs are shared out over the CTA: wide CTAs while the
      // grid leaves SMs free (measured on the 7x7 and 5x10 plans: 512
      // threads 14 % and 33 % faster than 128), narrow ones when many CTAs
      // share each SM
      const int64_t ctas = (int64_t)nsub * nb;
      const int sub_threads = ctas < 2 * (int64_t)sm_count ? 512 : (ctas < 4 * (int64_t)sm_count ? 256 : 128);
      (void)launch_chained(k_tree_subtrees, dim3(nsub, nb), dim3(sub_threads), sub_smem, st, a, d_subs, d_sleaves,
                           d_ssteps, d_slev);
      if (rec) cudaEventRecord(ev[1], st);
      last_launches++;
      TDQ_CUDA_TRY(cudaGetLastError());
      const bool conc = !rec && !side.empty();
      if (conc) {
        TDQ_CUDA_TRY(cudaEventRecord(fork_ev, st));
        for (cudaStream_t x : side) TDQ_CUDA_TRY(cudaStreamWaitEvent(x, fork_ev, 0));
      }
      for (int s = 0; s < nsteps; s++) {
        cudaStream_t ss = st;
        if (conc) {
          if (step_stream[s] > 0) ss = side[step_stream[s] - 1];
          for (int w : step_waits[s]) TDQ_CUDA_TRY(cudaStreamWaitEvent(ss, step_ev[w], 0));
        }
        if (rec) cudaEventRecord(ev[2 + 2 * s], st);
        const tdq_status ls = launch_step(a, s, nb, ss);
        if (ls != TDQ_OK) return ls;
        if (rec) cudaEventRecord(ev[3 + 2 * s], st);
        if (conc && step_ev[s]) TDQ_CUDA_TRY(cudaEventRecord(step_ev[s], ss));
        last_launches++;
      }
      if (conc) {
        for (size_t k = 0; k < side.size(); k++) {
          TDQ_CUDA_TRY(cudaEventRecord(join_ev[k], side[k]));
          TDQ_CUDA_TRY(cudaStreamWaitEvent(st, join_ev[k], 0));
        }
      }
      if (root_off >= 0) {
        (void)launch_chained(k_tree_roots, dim3((nb + 255) / 256), dim3(256), 0, st, a);
        last_launches++;
      }
      (void)launch_chained(k_slice_sum, dim3((B + 127) / 128), dim3(128), 0, st, d_roots, B, a.chunk, d_acc,
                           s0 == s_lo);
      last_launches++;
      auto adj_blocks = [](const StepDev& sd) {
        const int64_t tot = ((int64_t)1 << (sd.nh + sd.nm + sd.nk)) + ((int64_t)1 << (sd.nh + sd.nn + sd.nk));
        return (unsigned)std::min<int64_t>((tot + 255) / 256, 4096);
      };
      if (adj == 2) {  // plain reverse tree: one launch per step, every value kept
        a.nleaves = nleaves_g;
        (void)launch_chained(k_tree_root_bar, dim3((nb + 127) / 128), dim3(128), 0, st, a);
        last_launches++;
        for (int s = nsteps - 1; s >= 0; s--) {
          (void)launch_chained(k_tree_step_adj, dim3(adj_blocks(steps_h[s]), nb), dim3(256), 0, st, a, s);
          last_launches++;
        }
        (void)launch_chained(k_tree_leaf_grads, dim3((unsigned)std::max(1, (nleaves_g * 3 + 127) / 128), nb),
                             dim3(128), 0, st, a);
        last_launches++;
        TDQ_CUDA_TRY(cudaGetLastError());
      }
      if (adj == 3) {  // recomputing reverse tree: region by region, root's region first
        a.nleaves = nleaves_g;
        (void)launch_chained(k_tree_root_bar, dim3((nb + 127) / 128), dim3(128), 0, st, a);
        last_launches++;
        TreeArgs ar = a;
        ar.steps = d_rsteps;
        for (size_t r = 0; r + 1 < reg_begin.size(); r++) {
          const int b0 = reg_begin[r], b1 = reg_begin[r + 1];
          for (int i = b0; i < b1 - 1; i++) {  // its values again (the root is a checkpoint)
            const tdq_status ls = launch_step_of(ar, i, nb, st, rsteps_h, d_rsteps, rstep_kind);
            if (ls != TDQ_OK) return ls;
            last_launches++;
          }
          for (int i = b1 - 1; i >= b0; i--) {
            (void)launch_chained(k_tree_step_adj, dim3(adj_blocks(rsteps_h[i]), nb), dim3(256), 0, st, ar, i);
            last_launches++;
          }
        }
        (void)launch_chained(k_tree_leaf_grads, dim3((unsigned)std::max(1, (nleaves_g * 3 + 127) / 128), nb),
                             dim3(128), 0, st, a);
        last_launches++;
        TDQ_CUDA_TRY(cudaGetLastError());
      }
    }
    (void)launch_chained(k_tree_out, dim3((B + 127) / 128), dim3(128), 0, st, d_acc, B, output, coeff, values);
    last_launches++;
    if (adj) {
      const int n = B * std::max(1, P);
      (void)launch_chained(k_tree_grads_out, dim3((n + 255) / 256), dim3(256), 0, st, d_gacc, n, grads);
      last_launches++;
    }
    TDQ_CUDA_TRY(cudaGetLastError());
    return ok();
  }

  tdq_status set_slice_range(int64_t first, int64_t count) override {
    if (first < 0 || count < 0 || first > n_slices || count > n_slices - first)
      return fail(TDQ_ERR_ARG, "tdq_exec_set_slice_range: range outside [0, " + std::to_string(n_slices) + ")");
    slice_lo = first;
    slice_hi = first + count;
    graph.reset();  // a captured graph ran the previous range
    return ok();
  }

  tdq_status status() override {
    TDQ_CUDA_TRY(cudaSetDevice(dev));
    TDQ_CUDA_TRY(cudaStreamSynchronize(last_stream));
    int h = 0;
    TDQ_CUDA_TRY(cudaMemcpy(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost));
    TDQ_CUDA_TRY(cudaMemset(d_status, 0, sizeof(int)));
    if (h & (1 << TDQ_ERR_NONFINITE)) return fail(TDQ_ERR_NONFINITE, "non-finite parameter or input");
    return ok();
  }

  int launches() const override { return last_launches; }

  tdq_status config(int* c4) const override {
    c4[0] = adj;  // reverse tree: 0 none, 1 fused, 2 every value kept, 3 recomputed by regions
    c4[1] = reg_begin.empty() ? 0 : (int)reg_begin.size() - 1;
    c4[2] = chunk;
    c4[3] = (int)std::min<int64_t>(arena, INT32_MAX);
    return ok();
  }

  void work(double* f, double* by, int* k) const override {
    *f = flops_row;
    *by = bytes_row;
    *k = nsteps > 0 ? 3 : 4;
  }

  tdq_status timings(float* ms, int max, int* n) override {
    if (ev.empty()) return fail(TDQ_ERR_STATE, "tdq_exec_timings: compiled without record_timings");
    const int units = (int)ev.size() / 2;
    if (n) *n = units;
    if (!ms) return ok();
    if (max < units) return fail(TDQ_ERR_ARG, "tdq_exec_timings: buffer too small");
    TDQ_CUDA_TRY(cudaSetDevice(dev));
    TDQ_CUDA_TRY(cudaStreamSynchronize(last_stream));
    for (int u = 0; u < units; u++) TDQ_CUDA_TRY(cudaEventElapsedTime(&ms[u], ev[2 * u], ev[2 * u + 1]));
    return ok();
  }
};

// First-fit arena over a sequence of allocations and releases.
constexpr int64_t kArenaAlign = 32;  // HBM arena block granularity (complex elements)

struct Arena {
  struct Blk {
    int64_t off, len;
  };
  std::vector<Blk> live;
  int64_t peak = 0;
  // block granularity in elements: the HBM arena uses 32 complex elements
  // (256 bytes), so that every tensor, and so every operand row block of the
  // tensor-core product, starts on a 16-byte boundary
  int64_t align = 1;
  int64_t alloc(int64_t len) {
    len = (len + align - 1) / align * align;
    int64_t pos = 0;
    size_t at = 0;
    for (; at < live.size(); at++) {
      if (live[at].off - pos >= len) break;
      pos = live[at].off + live[at].len;
    }
    live.insert(live.begin() + at, {pos, len});
    peak = std::max(peak, pos + len);
    return pos;
  }
  void release(int64_t o) {
    for (size_t i = 0; i < live.size(); i++)
      if (live[i].off == o) {
        live.erase(live.begin() + i);
        return;
      }
  }
};

}  // namespace tdq

using namespace tdq;

// Steps whose three tensors all have at most 2^small_log2 entries (default
// kSmallLog2) and whose inputs come from leaves or such steps run inside
// subtree CTAs.
static constexpr int kSmallLog2 = 11;

// Which tensors are made inside subtree CTAs (leaves always are).
static std::vector<char> subtree_members(const Plan& plan, const std::vector<std::vector<int>>& T, int nl,
                                         bool plain, int small_log2 = kSmallLog2) {
  std::vector<char> in_sub(T.size(), 0);
  for (int t = 0; t < nl; t++) in_sub[t] = 1;
  const int lim = plain ? -1 : small_log2;  // the plain form: every step its own launch
  for (size_t s = 0; s < plan.steps.size(); s++) {
    const int a = plan.steps[s].a, b = plan.steps[s].b, c = nl + (int)s;
    const bool small = (int)T[a].size() <= lim && (int)T[b].size() <= lim && (int)T[c].size() <= lim;
    in_sub[c] = small && in_sub[a] && in_sub[b];
  }
  return in_sub;
}

// Kernel of a large step: 0 thread per entry, 1 SIMT tiled, 2 tensor core (A as
// X), 3 tensor core (B as X), 4 warp per entry, 5 split k.  Steps below
// 2^tc_min_log2 complex multiply-adds stay off the tensor cores (default: none;
// measured on the 7x7 amplitude plans, the tensor-core product beats the SIMT
// tiles at every size its 128 x 64 tiles fit).
static constexpr int kTcMinLog2 = 1;
static int large_step_kind(int nm, int nn, int nk, bool plain, int tc_min_log2 = kTcMinLog2, int nh = 0) {
  int kind = nm >= 6 && nn >= 6 && nk >= 4 ? 1 : (nk >= 6 ? 4 : 0);
  // wide outputs over a short k: the shared-memory tiles still give every
  // operand row to 64 outputs (a thread per output re-reads them)
  if (kind == 0 && nm + nn >= 15 && std::min(nm, nn) >= 4) kind = 1;
  // few outputs over a long k: split k across CTAs (operand chunks staged once)
  if (kind == 4 && nh + nm + nn <= 12 && nk >= 8) kind = 5;
  // tcgen05 tiles: 128 rows of X, 64 of Y, k in blocks of 8; one launch per
  // value of the hyperedge bits, so at most 4 of them
  if (!plain && nk >= 3 && nh <= 2 && nh + nm + nn + nk >= tc_min_log2) {
    if (nm >= 7 && nn >= 6) kind = 2;
    else if (nn >= 7 && nm >= 6) kind = 3;
  }
  return kind;
}

extern "C" tdq_status tdq_plan_compile(const tdq_plan* p, const tdq_compile_opts* o, tdq_exec** out) {
  if (!p || !o || !out) return fail(TDQ_ERR_ARG, "tdq_plan_compile: NULL argument");
  *out = nullptr;
  if (o->batch < 1) return fail(TDQ_ERR_ARG, "tdq_plan_compile: batch must be >= 1");
  if (o->grad != TDQ_GRAD_NONE && o->grad != TDQ_GRAD_ADJOINT)
    return fail(TDQ_ERR_UNSUPPORTED, "tdq_plan_compile: tree plans take adjoint gradients (or none)");
  if (o->grad == TDQ_GRAD_ADJOINT && p->plan.net->output != TDQ_OUT_EXPVAL)
    return fail(TDQ_ERR_UNSUPPORTED, "tdq_plan_compile: gradients need an expectation network");
  if (o->subtree_log2 < 0 || o->subtree_log2 > 13)
    return fail(TDQ_ERR_ARG, "tdq_plan_compile: subtree_log2 must be 0 (default) or 1..13");
  const int small_log2 = o->subtree_log2 > 0 ? o->subtree_log2 : kSmallLog2;
  if (o->tc_min_log2 < 0 || o->tc_min_log2 > 64)
    return fail(TDQ_ERR_ARG, "tdq_plan_compile: tc_min_log2 must be 0 (default) or 1..64");
  const int tc_min = o->tc_min_log2 > 0 ? o->tc_min_log2 : kTcMinLog2;
  const Plan& plan = p->plan;
  const Network& net = *plan.net;
  const int nl = (int)net.leaves.size();
  const int nst = (int)plan.steps.size();
  if (nst != nl - 1) return fail(TDQ_ERR_STATE, "tdq_plan_compile: incomplete path");
  if (plan.sliced.size() > 30) return fail(TDQ_ERR_UNSUPPORTED, "tdq_plan_compile: more than 30 sliced indices");
  auto T = ssa_indices(net, plan.steps, plan.sliced);
  const int ntens = (int)T.size();
  for (const auto& t : T)
    if (t.size() > 30) return fail(TDQ_ERR_UNSUPPORTED, "tdq_plan_compile: tensor wider than 2^30; slice it");
  if (!T.back().empty()) return fail(TDQ_ERR_STATE, "tdq_plan_compile: network has open indices");

  std::vector<int> consumer(ntens, -1);
  for (int s = 0; s < nst; s++) {
    consumer[plan.steps[s].a] = s;
    consumer[plan.steps[s].b] = s;
  }
  // storage order (most significant first): the consumer's hyperedge indices
  // (on both operands and its result), outer indices, then the ones it sums
  auto has = [](const std::vector<int>& v, int i) { return std::find(v.begin(), v.end(), i) != v.end(); };
  std::vector<std::vector<int>> order(ntens);
  for (int t = 0; t < ntens; t++) {
    if (consumer[t] < 0) continue;
    const Step& s = plan.steps[consumer[t]];
    const auto& other = T[s.a == t ? s.b : s.a];
    const auto& res = T[nl + consumer[t]];
    std::vector<int> hyp, outer, summed;
    for (int i : T[t]) {
      if (!has(other, i)) outer.push_back(i);
      else if (has(res, i)) hyp.push_back(i);
      else summed.push_back(i);
    }
    if ((int)hyp.size() > kMaxHyperBits)
      return fail(TDQ_ERR_UNSUPPORTED, "tdq_plan_compile: a step keeps more than 16 hyperedge indices");
    std::sort(hyp.begin(), hyp.end());
    std::sort(outer.begin(), outer.end());
    std::sort(summed.begin(), summed.end());
    order[t] = hyp;
    order[t].insert(order[t].end(), outer.begin(), outer.end());
    order[t].insert(order[t].end(), summed.begin(), summed.end());
  }
  auto bitpos = [&](int t, int id) {
    const auto& o2 = order[t];
    for (size_t i = 0; i < o2.size(); i++)
      if (o2[i] == id) return (int)(o2.size() - 1 - i);
    return -1;
  };
  // reverse tree: the whole network in one CTA when every step is small and
  // values plus cotangents fit in shared memory (fused), else every step its
  // own launch with every value kept (plain)
  bool plain = o->plain != 0;
  int adj_mode = 0;
  int64_t vt_total = 0;
  if (o->grad == TDQ_GRAD_ADJOINT) {
    const std::vector<char> all_small = subtree_members(plan, T, nl, false, small_log2);
    for (int t = 0; t < ntens; t++) vt_total += (int64_t)1 << T[t].size();
    const size_t need = sizeof(c2) * (size_t)(2 * vt_total + 2) + sizeof(StepDev) * (size_t)nst;
    if (!plain && all_small[ntens - 1] && need <= 200 * 1024) adj_mode = 1;
    else {
      adj_mode = 2;
      plain = true;
    }
  }
  // small steps (run inside subtree CTAs) and subtree membership
  const std::vector<char> in_sub = subtree_members(plan, T, nl, plain, small_log2);
  // subtree roots: tensors made inside a subtree but consumed outside one (or the network root)
  std::vector<int> roots;
  for (int t = 0; t < ntens; t++) {
    if (!in_sub[t]) continue;
    if (consumer[t] < 0 || !in_sub[nl + consumer[t]]) roots.push_back(t);
  }
  auto make_step = [&](int s, const std::vector<int64_t>& off) {
    const int a = plan.steps[s].a, b = plan.steps[s].b, c = nl + s;
    StepDev d{};
    d.a_off = off[a];
    d.b_off = off[b];
    d.c_off = off[c];
    int nk = 0, nh = 0;
    for (int i : T[a])
      if (has(T[b], i)) (has(T[c], i) ? nh : nk)++;
    d.nk = (int8_t)nk;
    d.nh = (int8_t)nh;
    d.nm = (int8_t)(T[a].size() - nk - nh);
    d.nn = (int8_t)(T[b].size() - nk - nh);
    d.rc = (int8_t)T[c].size();
    const auto& oa = order[a];
    const auto& ob = order[b];
    for (int i = 0; i < d.nm; i++) d.cm[i] = (int8_t)bitpos(c, oa[oa.size() - 1 - (nk + i)]);
    for (int i = 0; i < d.nn; i++) d.cn[i] = (int8_t)bitpos(c, ob[ob.size() - 1 - (nk + i)]);
    for (int i = 0; i < nh; i++) d.ch[i] = (int8_t)bitpos(c, oa[oa.size() - 1 - (nk + d.nm + i)]);
    return d;
  };
  auto make_leaf = [&](int t, int64_t off) {
    const Leaf& L = net.leaves[t];
    LeafDev d{};
    d.kind = (int8_t)L.kind;
    d.conj = (int8_t)L.conj;
    d.bit = (int8_t)L.bit;
    d.rank = (int8_t)T[t].size();
    d.rfull = (int8_t)L.idx.size();
    d.flip = (int8_t)L.flip;
    for (int j = 0; j < 3; j++) {
      d.src[j] = TDQ_FIXED;
      d.fixed[j] = 0.f;
    }
    d.gkind = -1;  // no gate (a state, bit or observable tensor)
    if (L.gate >= 0) {
      const GateRec& G = net.circ.gates[L.gate];
      d.gkind = (int8_t)G.kind;
      for (int j = 0; j < gate_n_angles(G.kind); j++) {
        d.src[j] = G.src[j];
        d.fixed[j] = (float)G.fixed[j];
      }
    }
    for (size_t q = 0; q < L.idx.size(); q++) {
      const int id = L.idx[q];
      auto it = std::find(plan.sliced.begin(), plan.sliced.end(), id);
      d.pos[q] = it != plan.sliced.end() ? (int8_t)(-1 - (int)(it - plan.sliced.begin())) : (int8_t)bitpos(t, id);
    }
    d.off = off;
    return d;
  };
  // the workspace budget (HBM), known before the reverse tree's layout is chosen
  if (cudaSetDevice(o->device) != cudaSuccess) return fail(TDQ_ERR_CUDA, "cudaSetDevice failed");
  size_t freeb = 0, totb = 0;
  cudaMemGetInfo(&freeb, &totb);
  const size_t budget = o->workspace_bytes > 0 ? (size_t)o->workspace_bytes
                                               : std::min<size_t>((size_t)64 << 30, freeb / 2);
  // global arena: subtree roots live from the start; large-step results from their step
  std::vector<int64_t> goff(ntens, -1);
  Arena ga;
  ga.align = kArenaAlign;
  for (int r : roots)
    if (consumer[r] >= 0) goff[r] = ga.alloc((int64_t)1 << T[r].size());
  std::vector<int> gsteps;
  for (int s = 0; s < nst; s++) {
    const int c = nl + s;
    if (in_sub[c]) continue;
    goff[c] = ga.alloc((int64_t)1 << T[c].size());
    if (adj_mode != 2) {  // the plain reverse tree reads every value again
      ga.release(goff[plan.steps[s].a]);
      ga.release(goff[plan.steps[s].b]);
    }
    gsteps.push_back(s);
  }
  // Reverse tree with recomputation, when keeping every value (plus its
  // cotangent) does not fit the budget: the forward pass keeps only the leaves
  // and the roots of regions of the tree (checkpoints); the reverse pass takes
  // the regions root first, recomputes a region's values from its checkpoints
  // into a scratch area, then runs its reverse steps.  A region grows down from
  // its root while its recomputed values stay within `cap` entries; an operand
  // that would exceed it becomes a checkpoint and the root of a new region.
  // The cap giving the smallest workspace is kept.  Cotangents mirror the
  // values at +boff, as in the other reverse modes.
  struct Region {
    int root;
    std::vector<int> steps;  // ascending: the last one makes the root
  };
  auto tsz = [&](int t) { return (int64_t)1 << T[t].size(); };
  auto aligned = [](int64_t n) { return (n + kArenaAlign - 1) / kArenaAlign * kArenaAlign; };
  auto regions_for = [&](int64_t cap, std::vector<char>& ck, std::vector<Region>& regs, std::vector<int64_t>& ckoff,
                         std::vector<int64_t>& fo, int64_t* ck_total, int64_t* scratch) {
    ck.assign(ntens, 0);
    regs.clear();
    for (int t = 0; t < nl; t++) ck[t] = 1;
    ck[ntens - 1] = 1;
    std::vector<int> q{ntens - 1};
    for (size_t qi = 0; qi < q.size(); qi++) {
      Region R;
      R.root = q[qi];
      int64_t acc = 0;
      std::vector<int> stack{R.root};
      while (!stack.empty()) {
        const int t = stack.back();
        stack.pop_back();
        const int st2 = t - nl;
        R.steps.push_back(st2);
        for (int u : {plan.steps[st2].a, plan.steps[st2].b}) {
          if (u < nl) continue;
          if (acc + aligned(tsz(u)) <= cap) {
            acc += aligned(tsz(u));
            stack.push_back(u);
          } else {
            ck[u] = 1;
            q.push_back(u);
          }
        }
      }
      std::sort(R.steps.begin(), R.steps.end());
      regs.push_back(std::move(R));
    }
    Arena ca;
    ca.align = kArenaAlign;
    ckoff.assign(ntens, -1);
    for (int t = 0; t < ntens; t++)
      if (ck[t]) ckoff[t] = ca.alloc(tsz(t));
    *ck_total = aligned(ca.peak);
    Arena fa;  // forward scratch: values that are not checkpoints, freed after their consumer
    fa.align = kArenaAlign;
    fo.assign(ntens, -1);
    for (int st2 = 0; st2 < nst; st2++) {
      const int c = nl + st2;
      if (!ck[c]) fo[c] = fa.alloc(tsz(c));
      for (int u : {plan.steps[st2].a, plan.steps[st2].b})
        if (!ck[u]) fa.release(fo[u]);
    }
    int64_t scr = fa.peak;
    for (const Region& R : regs) {  // a region keeps all its recomputed values
      int64_t sum = 0;
      for (int st2 : R.steps)
        if (!ck[nl + st2]) sum += aligned(tsz(nl + st2));
      scr = std::max(scr, sum);
    }
    *scratch = aligned(scr);
  };
  std::vector<char> rck;
  std::vector<Region> rregs;
  std::vector<int64_t> rckoff, rfo;
  int64_t rck_total = 0;
  if (adj_mode == 2 && sizeof(c2) * 2 * (size_t)ga.peak * (size_t)o->batch > budget) {
    int64_t best = -1, best_cap = 0;
    for (int j = 0; j <= 40; j++) {
      int64_t ckt = 0, scr = 0;
      regions_for((int64_t)1 << j, rck, rregs, rckoff, rfo, &ckt, &scr);
      if (best < 0 || ckt + scr < best) {
        best = ckt + scr;
        best_cap = (int64_t)1 << j;
      }
    }
    if (sizeof(c2) * 2 * (size_t)best * (size_t)o->batch <= budget) {
      int64_t scr = 0;
      regions_for(best_cap, rck, rregs, rckoff, rfo, &rck_total, &scr);
      adj_mode = 3;
      ga.peak = rck_total + scr;
      for (int t = 0; t < ntens; t++) goff[t] = rck[t] ? rckoff[t] : (rfo[t] >= 0 ? rck_total + rfo[t] : -1);
    }
  }
  // subtrees: leaves and steps level by level, shared arena planned per subtree
  std::vector<LeafDev> sleaves;
  std::vector<StepDev> ssteps;
  std::vector<SubDev> subs;
  std::vector<int> slev;  // level bounds of every subtree (relative step indices)
  size_t max_smem = 0;
  std::vector<int> owner(ntens, -1);
  for (size_t ri = 0; ri < roots.size(); ri++) {  // mark members
    std::vector<int> stack{roots[ri]};
    while (!stack.empty()) {
      const int t = stack.back();
      stack.pop_back();
      owner[t] = (int)ri;
      if (t >= nl) {
        stack.push_back(plan.steps[t - nl].a);
        stack.push_back(plan.steps[t - nl].b);
      }
    }
  }
  std::vector<int> lev(ntens, 0);  // level of a subtree member: 0 for leaves, 1 + its operands' highest
  for (int s = 0; s < nst; s++)
    if (owner[nl + s] >= 0) lev[nl + s] = 1 + std::max(lev[plan.steps[s].a], lev[plan.steps[s].b]);
  for (size_t ri = 0; ri < roots.size(); ri++) {
    std::vector<int> members;  // the subtree's steps in path order
    for (int s = 0; s < nst; s++)
      if (owner[nl + s] == (int)ri) members.push_back(s);
    // Shared arena: leaves first, then the steps level by level (every output
    // of a level allocated before any of its operands is released, so the
    // steps of a level never overlap each other's operands); if that needs
    // more than twice the arena of the one-step-at-a-time plan (or more than
    // the shared memory allows), the steps run one per level instead.
    auto plan_arena = [&](bool by_level, std::vector<int64_t>& loff, std::vector<std::vector<int>>& levels) {
      Arena sa;
      loff.assign(ntens, -1);
      levels.clear();
      for (int t = 0; t < nl; t++)
        if (owner[t] == (int)ri) loff[t] = sa.alloc((int64_t)1 << T[t].size());
      if (by_level) {
        int top = 0;
        for (int s : members) top = std::max(top, lev[nl + s]);
        levels.assign(top, {});
        for (int s : members) levels[lev[nl + s] - 1].push_back(s);
      } else {
        for (int s : members) levels.push_back({s});
      }
      for (const auto& L : levels) {
        for (int s : L) loff[nl + s] = sa.alloc((int64_t)1 << T[nl + s].size());
        for (int s : L) {
          sa.release(loff[plan.steps[s].a]);
          sa.release(loff[plan.steps[s].b]);
        }
      }
      return sa.peak;
    };
    std::vector<int64_t> loff, loff1;
    std::vector<std::vector<int>> levels, levels1;
    const int64_t peak1 = plan_arena(false, loff1, levels1);
    int64_t peak = plan_arena(true, loff, levels);
    if (peak > 2 * peak1 || sizeof(c2) * (size_t)peak + sizeof(StepDev) * members.size() > 160 * 1024) {
      peak = peak1;
      loff = loff1;
      levels = levels1;
    }
    SubDev sd{};
    sd.leaf_begin = (int)sleaves.size();
    for (int t = 0; t < nl; t++)
      if (owner[t] == (int)ri) sleaves.push_back(make_leaf(t, loff[t]));
    sd.leaf_end = (int)sleaves.size();
    sd.step_begin = (int)ssteps.size();
    sd.lev_begin = (int)slev.size();
    sd.nlev = (int)levels.size();
    slev.push_back(0);
    for (const auto& L : levels) {
      uint32_t pre = 0;
      for (int s : L) {
        StepDev d = make_step(s, loff);
        d.pre = pre;
        pre += 1u << (d.nm + d.nn + d.nh);
        ssteps.push_back(d);
      }
      slev.push_back((int)ssteps.size() - sd.step_begin);
    }
    sd.step_end = (int)ssteps.size();
    // every tensor of this subtree's steps inside its shared arena, and within
    // a level no output overlapping another output or any operand of the level
    for (int st = 0; st < nst; st++) {
      if (owner[nl + st] != (int)ri) continue;
      for (int t : {plan.steps[st].a, plan.steps[st].b, nl + st})
        if (loff[t] < 0 || loff[t] + ((int64_t)1 << T[t].size()) > peak)
          return fail(TDQ_ERR_STATE, "tdq_plan_compile: a subtree step leaves its shared arena");
    }
    auto span = [&](int t) { return std::make_pair(loff[t], loff[t] + ((int64_t)1 << T[t].size())); };
    auto overlap = [](std::pair<int64_t, int64_t> x, std::pair<int64_t, int64_t> y) {
      return x.first < y.second && y.first < x.second;
    };
    for (const auto& L : levels)
      for (int x : L)
        for (int y : L) {
          const auto ox = span(nl + x);
          if ((x != y && overlap(ox, span(nl + y))) || overlap(ox, span(plan.steps[y].a)) ||
              overlap(ox, span(plan.steps[y].b)))
            return fail(TDQ_ERR_STATE, "tdq_plan_compile: subtree steps of one level overlap");
        }
    sd.smem_elems = (int)((peak + 1) & ~(int64_t)1);  // keep the step table 16-byte aligned
    sd.root_local = (int)loff[roots[ri]];
    sd.root_size = 1 << T[roots[ri]].size();
    sd.root_global = consumer[roots[ri]] >= 0 ? goff[roots[ri]] : -1;
    subs.push_back(sd);
    max_smem = std::max(max_smem, sizeof(c2) * (size_t)sd.smem_elems +
                                      sizeof(StepDev) * (size_t)(sd.step_end - sd.step_begin));
  }
  if (max_smem > 200 * 1024)
    return fail(TDQ_ERR_UNSUPPORTED, "tdq_plan_compile: a subtree's shared arena exceeds 200 KiB");

  TreeExec* e = new (std::nothrow) TreeExec();
  if (!e) return fail(TDQ_ERR_OOM, "tdq_plan_compile: host allocation");
  auto bail = [&](tdq_status st) {
    delete e;
    return st;
  };
  e->dev = o->device;
  e->B = o->batch;
  e->P = net.circ.n_params;
  e->F = net.circ.n_inputs;
  e->output = net.output;
  e->coeff = net.coeff;
  e->plain = plain;
  e->n_sliced = (int)plan.sliced.size();
  e->n_slices = (int64_t)1 << e->n_sliced;
  e->arena = std::max<int64_t>(ga.peak, 1);
  e->adj = adj_mode;
  if (adj_mode == 2 || adj_mode == 3) {  // cotangents mirror the values
    e->boff = e->arena;
    e->arena *= 2;
  }
  e->root_off = in_sub[ntens - 1] ? -1 : goff[ntens - 1];
  e->nsub = (int)subs.size();
  e->sub_smem = max_smem;
  if (cudaDeviceGetAttribute(&e->sm_count, cudaDevAttrMultiProcessorCount, o->device) != cudaSuccess)
    return bail(fail(TDQ_ERR_CUDA, "tdq_plan_compile: cudaDeviceGetAttribute failed"));
  double flops = 0, bytes = 0;
  for (int s = 0; s < nst; s++) {
    const int a = plan.steps[s].a, b = plan.steps[s].b, c = nl + s;
    int nk = 0;  // summed indices: on both operands, not on the result
    for (int i : T[a])
      if (has(T[b], i) && !has(T[c], i)) nk++;
    // complex MACs (2^(|C| + summed)): 8 real FLOPs each; bytes: both operands read, result written
    flops += 8.0 * std::ldexp(1.0, (int)T[c].size() + nk);
    if (!in_sub[c])
      bytes += 8.0 * (std::ldexp(1.0, (int)T[a].size()) + std::ldexp(1.0, (int)T[b].size()) +
                      std::ldexp(1.0, (int)T[c].size()));
  }
  e->flops_row = flops * (double)e->n_slices;
  e->bytes_row = bytes * (double)e->n_slices;
  for (int s : gsteps) {
    StepDev d = make_step(s, goff);
    // every operand and the result inside the workspace (the value half)
    for (int t : {plan.steps[s].a, plan.steps[s].b, nl + s})
      if (goff[t] < 0 || goff[t] + ((int64_t)1 << T[t].size()) > (e->adj >= 2 ? e->boff : e->arena))
        return bail(fail(TDQ_ERR_STATE, "tdq_plan_compile: step " + std::to_string(s) + " leaves the workspace"));
    e->steps_h.push_back(d);
    e->step_kind.push_back(large_step_kind(d.nm, d.nn, d.nk, plain, tc_min, d.nh));
  }
  e->nsteps = (int)gsteps.size();
  // Concurrent schedule of the large steps (values only; timed and plain runs
  // stay in path order on one stream).  Step i waits for the producers of its
  // operands and for every earlier step that reads or writes arena space its
  // result reuses; chains of the tree stay on one stream, independent branches
  // take other streams.
  std::vector<std::vector<int>> deps(e->nsteps);
  int n_side = 0;
  if (!plain && adj_mode == 0 && !o->record_timings && e->nsteps > 1) {
    std::vector<int> gidx(nst, -1);
    for (int i = 0; i < e->nsteps; i++) gidx[gsteps[i]] = i;
    auto overlap = [&](int t, int u) {
      const int64_t a0 = goff[t], a1 = a0 + ((int64_t)1 << T[t].size());
      const int64_t b0 = goff[u], b1 = b0 + ((int64_t)1 << T[u].size());
      return a0 < b1 && b0 < a1;
    };
    std::vector<std::vector<int>> prod(e->nsteps);
    for (int i = 0; i < e->nsteps; i++) {
      const int st = gsteps[i], c = nl + st;
      for (int t : {plan.steps[st].a, plan.steps[st].b})
        if (t >= nl && gidx[t - nl] >= 0) prod[i].push_back(gidx[t - nl]);
      deps[i] = prod[i];
      for (int j = 0; j < i; j++) {
        const int sj = gsteps[j];
        for (int t : {plan.steps[sj].a, plan.steps[sj].b, nl + sj})
          if (goff[t] >= 0 && overlap(t, c)) {
            deps[i].push_back(j);
            break;
          }
      }
      std::sort(deps[i].begin(), deps[i].end());
      deps[i].erase(std::unique(deps[i].begin(), deps[i].end()), deps[i].end());
    }
    constexpr int kStreams = 4;
    std::vector<int> sid(e->nsteps, 0), tail(kStreams, -1);
    int nstreams = 0;
    for (int i = 0; i < e->nsteps; i++) {
      int pick = -1;
      for (int d : prod[i])
        if (tail[sid[d]] == d) {
          pick = sid[d];
          break;
        }
      if (pick < 0) {
        if (nstreams < kStreams) {
          pick = nstreams++;
        } else {
          pick = 0;
          for (int k = 1; k < kStreams; k++)
            if (tail[k] < tail[pick]) pick = k;
        }
      }
      sid[i] = pick;
      tail[pick] = i;
    }
    e->step_stream = sid;
    e->step_waits.assign(e->nsteps, {});
    e->step_ev.assign(e->nsteps, nullptr);
    for (int i = 0; i < e->nsteps; i++)
      for (int d : deps[i])
        if (sid[d] != sid[i]) e->step_waits[i].push_back(d);
    n_side = nstreams - 1;
    // Race check of the schedule: steps i < j with no order between them (no
    // path of dependencies, and on different streams) must not touch the same
    // workspace where either writes.  Order: same stream, or a chain of waits.
    const int n = e->nsteps, words = (n + 63) / 64;
    std::vector<uint64_t> before((size_t)n * words, 0);  // before[j]: steps ordered before j
    std::vector<int> last_on(kStreams, -1);
    for (int j = 0; j < n; j++) {
      uint64_t* bj = &before[(size_t)j * words];
      auto take = [&](int d) {
        bj[d / 64] |= 1ull << (d % 64);
        const uint64_t* bd = &before[(size_t)d * words];
        for (int w = 0; w < words; w++) bj[w] |= bd[w];
      };
      if (last_on[sid[j]] >= 0) take(last_on[sid[j]]);
      for (int d : deps[j]) take(d);
      last_on[sid[j]] = j;
    }
    auto span = [&](int t) { return std::make_pair(goff[t], goff[t] + ((int64_t)1 << T[t].size())); };
    auto meet = [](std::pair<int64_t, int64_t> x, std::pair<int64_t, int64_t> y) {
      return x.first < y.second && y.first < x.second;
    };
    for (int j = 0; j < n; j++)
      for (int i = 0; i < j; i++) {
        if (before[(size_t)j * words + i / 64] >> (i % 64) & 1) continue;
        const Step& si = plan.steps[gsteps[i]];
        const Step& sj = plan.steps[gsteps[j]];
        const auto wi = span(nl + gsteps[i]), wj = span(nl + gsteps[j]);
        bool clash = meet(wi, wj) || meet(wi, span(sj.a)) || meet(wi, span(sj.b)) || meet(wj, span(si.a)) ||
                     meet(wj, span(si.b));
        if (clash)
          return bail(fail(TDQ_ERR_STATE, "tdq_plan_compile: concurrent steps " + std::to_string(i) + " and " +
                                              std::to_string(j) + " would race on the workspace"));
      }
  }
  if (cudaSetDevice(e->dev) != cudaSuccess) return bail(fail(TDQ_ERR_CUDA, "cudaSetDevice failed"));
  if (!plain && adj_mode == 0 && !o->record_timings) {
    const tdq_status gs = e->graph.init();
    if (gs != TDQ_OK) return bail(gs);
    e->use_graph = true;
  }
  if (n_side > 0) {
    for (int i = 0; i < e->nsteps; i++)
      for (int d : e->step_waits[i])
        if (!e->step_ev[d] && cudaEventCreateWithFlags(&e->step_ev[d], cudaEventDisableTiming) != cudaSuccess)
          return bail(fail(TDQ_ERR_CUDA, "tdq_plan_compile: event"));
    if (cudaEventCreateWithFlags(&e->fork_ev, cudaEventDisableTiming) != cudaSuccess)
      return bail(fail(TDQ_ERR_CUDA, "tdq_plan_compile: event"));
    for (int k = 0; k < n_side; k++) {
      cudaStream_t x;
      cudaEvent_t j;
      if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(TDQ_ERR_CUDA, "tdq_plan_compile: stream"));
      e->side.push_back(x);
      if (cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(TDQ_ERR_CUDA, "tdq_plan_compile: event"));
      e->join_ev.push_back(j);
    }
  }
  auto up = [&](void** d, const void* h, size_t bytes2) -> tdq_status {
    if (bytes2 == 0) return TDQ_OK;
    if (cudaMalloc(d, bytes2) != cudaSuccess) return fail(TDQ_ERR_OOM, "tdq_plan_compile: cudaMalloc");
    if (cudaMemcpy(*d, h, bytes2, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(TDQ_ERR_CUDA, "tdq_plan_compile: cudaMemcpy");
    return TDQ_OK;
  };
  tdq_status s;
  if ((s = up((void**)&e->d_sleaves, sleaves.data(), sizeof(LeafDev) * sleaves.size())) != TDQ_OK) return bail(s);
  if ((s = up((void**)&e->d_ssteps, ssteps.data(), sizeof(StepDev) * ssteps.size())) != TDQ_OK) return bail(s);
  if ((s = up((void**)&e->d_subs, subs.data(), sizeof(SubDev) * subs.size())) != TDQ_OK) return bail(s);
  if ((s = up((void**)&e->d_slev, slev.data(), sizeof(int) * slev.size())) != TDQ_OK) return bail(s);
  if ((s = up((void**)&e->d_steps, e->steps_h.data(), sizeof(StepDev) * e->steps_h.size())) != TDQ_OK)
    return bail(s);
  if (cudaFuncSetAttribute(k_tree_subtrees, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem) !=
      cudaSuccess)
    return bail(fail(TDQ_ERR_CUDA, "tdq_plan_compile: shared memory attribute"));
  const size_t per = sizeof(c2) * (size_t)e->arena * (size_t)e->B;
  if (per > budget)
    return bail(fail(TDQ_ERR_OOM, "tdq_plan_compile: one slice of the batch exceeds the workspace budget; slice further"));
  if (e->B > 65535) return bail(fail(TDQ_ERR_UNSUPPORTED, "tdq_plan_compile: batch above 65535"));
  e->chunk = (int)std::max<int64_t>(1, std::min<int64_t>(e->n_slices, (int64_t)(budget / per)));
  e->chunk = std::max(1, std::min(e->chunk, 65535 / e->B));  // batch entries ride on grid.y / grid.z
  if (plain) e->chunk = 1;  // the plain form: one slice at a time
  if (cudaMalloc(&e->d_work, per * e->chunk) != cudaSuccess)
    return bail(fail(TDQ_ERR_OOM, "tdq_plan_compile: workspace"));
  if (cudaMalloc(&e->d_roots, sizeof(c2) * (size_t)e->B * e->chunk) != cudaSuccess ||
      cudaMalloc(&e->d_acc, sizeof(double) * 2 * e->B) != cudaSuccess ||
      cudaMalloc(&e->d_status, sizeof(int)) != cudaSuccess)
    return bail(fail(TDQ_ERR_OOM, "tdq_plan_compile: buffers"));
  cudaMemset(e->d_status, 0, sizeof(int));
  if (adj_mode) {
    if (cudaMalloc(&e->d_gacc, sizeof(double) * (size_t)e->B * std::max(1, e->P)) != cudaSuccess)
      return bail(fail(TDQ_ERR_OOM, "tdq_plan_compile: gradient buffer"));
  }
  if (adj_mode == 2 || adj_mode == 3) {
    std::vector<LeafDev> gl;
    for (int t = 0; t < nl; t++) gl.push_back(make_leaf(t, goff[t]));
    if ((s = up((void**)&e->d_gleaves, gl.data(), sizeof(LeafDev) * gl.size())) != TDQ_OK) return bail(s);
    e->nleaves_g = nl;
  }
  if (adj_mode == 3) {  // each region's steps: checkpoints at their fixed offsets, the rest in the scratch
    for (const Region& R : rregs) {
      std::vector<int64_t> off(ntens, -1);
      for (int t = 0; t < ntens; t++)
        if (rck[t]) off[t] = rckoff[t];
      int64_t bump = rck_total;
      for (int st2 : R.steps)
        if (!rck[nl + st2]) {
          off[nl + st2] = bump;
          bump += aligned(tsz(nl + st2));
        }
      e->reg_begin.push_back((int)e->rsteps_h.size());
      for (int st2 : R.steps) {
        StepDev d = make_step(st2, off);
        e->rsteps_h.push_back(d);
        e->rstep_kind.push_back(large_step_kind(d.nm, d.nn, d.nk, true, tc_min, d.nh));
      }
    }
    e->reg_begin.push_back((int)e->rsteps_h.size());
    if ((s = up((void**)&e->d_rsteps, e->rsteps_h.data(), sizeof(StepDev) * e->rsteps_h.size())) != TDQ_OK)
      return bail(s);
  }
  if (adj_mode == 1) {
    std::vector<int64_t> vo(ntens, 0);
    int64_t cur = 0;
    for (int t = 0; t < ntens; t++) {
      vo[t] = cur;
      cur += (int64_t)1 << T[t].size();
    }
    std::vector<LeafDev> fl;
    std::vector<StepDev> fs;
    for (int t = 0; t < nl; t++) fl.push_back(make_leaf(t, vo[t]));
    for (int s2 = 0; s2 < nst; s2++) fs.push_back(make_step(s2, vo));
    e->nfleaves = nl;
    e->nfsteps = nst;
    e->froot = (int)vo[ntens - 1];
    e->boff = vt_total;
    e->fsmem_elems = (int)((2 * vt_total + 1) & ~(int64_t)1);
    e->fsmem = sizeof(c2) * (size_t)e->fsmem_elems + sizeof(StepDev) * (size_t)nst;
    if ((s = up((void**)&e->d_fleaves, fl.data(), sizeof(LeafDev) * fl.size())) != TDQ_OK) return bail(s);
    if ((s = up((void**)&e->d_fsteps, fs.data(), sizeof(StepDev) * fs.size())) != TDQ_OK) return bail(s);
    if (cudaFuncSetAttribute(k_tree_fused_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->fsmem) !=
        cudaSuccess)
      return bail(fail(TDQ_ERR_CUDA, "tdq_plan_compile: shared memory attribute"));
  }
  if (o->record_timings) {
    e->ev.resize(2 * (1 + e->nsteps));
    for (auto& x : e->ev)
      if (cudaEventCreate(&x) != cudaSuccess) return bail(fail(TDQ_ERR_CUDA, "tdq_plan_compile: event"));
  }
  *out = e;
  return ok();
}

// Launch units of a compiled plan and their features (same partition as
// tdq_plan_compile): unit 0 is the subtree launch, then one unit per large
// step.  Features (kTdqFeatures per unit, all log2 unless marked):
//   0..5 one-hot kind: subtrees, thread/entry, SIMT tiled, tensor core, warp/entry, (spare)
//   6 rows (larger outer side)  7 cols (smaller outer side)  8 k
//   9 batch entries per launch  10 FLOPs  11 bytes moved
// For the subtree unit: 6 subtrees, 7 largest subtree (steps), 8 small steps.
static constexpr int kTdqFeatures = 12;

extern "C" tdq_status tdq_plan_features(const tdq_plan* p, int batch, int64_t workspace_bytes, float* feats,
                                        int max_units, int* n_units, int* repeats) {
  if (!p || batch < 1) return fail(TDQ_ERR_ARG, "tdq_plan_features: bad argument");
  const Plan& plan = p->plan;
  const Network& net = *plan.net;
  const int nl = (int)net.leaves.size(), nst = (int)plan.steps.size();
  if (nst != nl - 1) return fail(TDQ_ERR_STATE, "tdq_plan_features: incomplete path");
  auto T = ssa_indices(net, plan.steps, plan.sliced);
  const std::vector<char> in_sub = subtree_members(plan, T, nl, false);
  std::vector<int> consumer(T.size(), -1);
  for (int s = 0; s < nst; s++) consumer[plan.steps[s].a] = consumer[plan.steps[s].b] = s;
  // global arena peak (for the slice batch size)
  struct A2 {
    std::vector<std::pair<int64_t, int64_t>> live;
    int64_t peak = 0;
    int64_t alloc(int64_t len) {
      len = (len + kArenaAlign - 1) / kArenaAlign * kArenaAlign;  // as the compiled arena
      int64_t pos = 0;
      size_t at = 0;
      for (; at < live.size(); at++) {
        if (live[at].first - pos >= len) break;
        pos = live[at].first + live[at].second;
      }
      live.insert(live.begin() + at, {pos, len});
      peak = std::max(peak, pos + len);
      return pos;
    }
    void release(int64_t o) {
      for (size_t i = 0; i < live.size(); i++)
        if (live[i].first == o) {
          live.erase(live.begin() + i);
          return;
        }
    }
  } ga;
  std::vector<int64_t> goff(T.size(), -1);
  int nsub = 0;
  for (size_t t = 0; t < T.size(); t++)
    if (in_sub[t] && (consumer[t] < 0 || !in_sub[nl + consumer[t]])) {
      nsub++;
      if (consumer[t] >= 0) goff[t] = ga.alloc((int64_t)1 << T[t].size());
    }
  std::vector<int> gsteps;
  for (int s = 0; s < nst; s++) {
    if (in_sub[nl + s]) continue;
    goff[nl + s] = ga.alloc((int64_t)1 << T[nl + s].size());
    ga.release(goff[plan.steps[s].a]);
    ga.release(goff[plan.steps[s].b]);
    gsteps.push_back(s);
  }
  const int64_t n_slices = (int64_t)1 << plan.sliced.size();
  const int64_t budget = workspace_bytes > 0 ? workspace_bytes : ((int64_t)64 << 30);
  const int64_t per = 8 * std::max<int64_t>(ga.peak, 1) * batch;
  int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n_slices, budget / std::max<int64_t>(per, 1)));
  chunk = std::max<int64_t>(1, std::min<int64_t>(chunk, 65535 / batch));
  const double nb = (double)batch * (double)chunk;
  const int units = 1 + (int)gsteps.size();
  if (n_units) *n_units = units;
  if (repeats) *repeats = (int)((n_slices + chunk - 1) / chunk);
  if (!feats) return ok();
  if (max_units < units) return fail(TDQ_ERR_ARG, "tdq_plan_features: buffer too small");
  std::fill(feats, feats + (size_t)units * kTdqFeatures, 0.f);
  // summed (k) and kept-shared hyperedge (h) indices of a step
  auto kh_of = [&](int s, int* nh) {
    const auto& A = T[plan.steps[s].a];
    const auto& B = T[plan.steps[s].b];
    const auto& C = T[nl + s];
    int nk = 0, h = 0;
    for (int i : A)
      if (std::find(B.begin(), B.end(), i) != B.end())
        (std::find(C.begin(), C.end(), i) != C.end() ? h : nk)++;
    if (nh) *nh = h;
    return nk;
  };
  // subtree unit
  {
    float* f = feats;
    double small_flops = 0, small_bytes = 0;
    int small_steps = 0;
    std::vector<int> sub_steps(T.size(), 0);  // steps inside the subtree of tensor t
    int largest = 0;
    for (int s = 0; s < nst; s++) {
      const int c = nl + s;
      if (!in_sub[c]) continue;
      const int a = plan.steps[s].a, b = plan.steps[s].b, nk = kh_of(s, nullptr);
      small_steps++;
      small_flops += 8.0 * std::ldexp(1.0, (int)T[c].size() + nk);
      small_bytes += 8.0 * (std::ldexp(1.0, (int)T[a].size()) + std::ldexp(1.0, (int)T[b].size()) +
                            std::ldexp(1.0, (int)T[c].size()));
      sub_steps[c] = 1 + sub_steps[a] + sub_steps[b];
      largest = std::max(largest, sub_steps[c]);
    }
    f[0] = 1.f;
    f[6] = (float)std::log2(1.0 + nsub);
    f[7] = (float)std::log2(1.0 + largest);
    f[8] = (float)std::log2(1.0 + small_steps);
    f[9] = (float)std::log2(nb);
    f[10] = (float)std::log2(1.0 + small_flops * nb);
    f[11] = (float)std::log2(1.0 + small_bytes * nb);
  }
  for (size_t u = 0; u < gsteps.size(); u++) {
    const int s = gsteps[u], a = plan.steps[s].a, b = plan.steps[s].b, c = nl + s;
    int nh = 0;
    const int nk = kh_of(s, &nh), nm = (int)T[a].size() - nk - nh, nn = (int)T[b].size() - nk - nh;
    const int kind = large_step_kind(nm, nn, nk, false, kTcMinLog2, nh);
    float* f = feats + (size_t)(u + 1) * kTdqFeatures;
    const int oh[6] = {1, 2, 3, 3, 4, 5};  // kind -> one-hot slot
    f[oh[kind]] = 1.f;
    f[6] = (float)std::max(nm, nn);
    f[7] = (float)std::min(nm, nn);
    f[8] = (float)nk;
    f[9] = (float)std::log2(nb) + (float)nh;  // hyperedge bits ride the batch
    f[10] = (float)std::log2(8.0 * nb) + (float)(nh + nm + nn + nk);
    f[11] = (float)std::log2(8.0 * nb * (std::ldexp(1.0, (int)T[a].size()) + std::ldexp(1.0, (int)T[b].size()) +
                                         std::ldexp(1.0, (int)T[c].size())));
  }
  return ok();
}
