// Kernel K1: tiled state sweep through HBM (see sweep_tiled.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "sweep_tiled.cuh"

namespace tdq {

namespace {

struct TiledDev {
  const SweepOp* ops;
  const int* off;      // this pass's 2^(k-L) offsets
  const int8_t* loc;   // this pass's 32 local-bit entries
  const RegPass* fp;   // this pass's forward register passes (ops relative to dop0)
  int nfp;
  const RegPass* bp;   // reverse register passes
  int nbp;
  const DOp* dops;     // this pass's decoded ops (forward then reverse)
  int ndops;
  int bo0, bo1;        // reverse ops range (relative)
  const int* rec_ptr;
  const int* rec_ops;
  int rec0, nrec;      // this pass's recipes
  c2* psi;
  c2* lam;
  double* gacc;
  double* vals;
  int n, k, L;
  uint32_t smask;
  int op_begin, op_end;
  int tiles_per_cta, ntiles;
  int row0;
};

// Spread the bits of t over the positions of mask (lowest first).
__device__ __forceinline__ uint32_t deposit(uint32_t t, uint32_t mask) {
  uint32_t out = 0;
  for (uint32_t m = mask; m && t; m &= m - 1, t >>= 1)
    if (t & 1u) out |= m & (0u - m);
  return out;
}

struct TileShared {
  c2* psi;
  c2* lam;
  OpMat* mats;    // [recipes of the pass]
  DOp* dops;      // [decoded ops of the pass]
  double* red;
  double* vsum;   // [n_groups]
  double* gpart;  // [3 * pass length]
  int* off;
  int8_t* loc;
};

// layout: psi[2^k] | lambda[2^k] (two) | mats[nrec] | dops[ndops] | red[32] | vsum[ng] |
//         gpart[3 nrec] | off[2^(k-L)] | loc[32]
__device__ __forceinline__ TileShared carve(unsigned char* raw, int k, int L, bool two, int nrec,
                                            int ndops, int ng) {
  TileShared s;
  const int nloc = 1 << k;
  const int npass = nrec;
  s.psi = reinterpret_cast<c2*>(raw);
  s.lam = s.psi + nloc;
  s.mats = reinterpret_cast<OpMat*>(s.psi + (two ? 2 : 1) * nloc);
  s.dops = reinterpret_cast<DOp*>(s.mats + nrec);
  s.red = reinterpret_cast<double*>(s.dops + ndops);
  s.vsum = s.red + 32;
  s.gpart = s.vsum + ng;
  s.off = reinterpret_cast<int*>(s.gpart + 3 * npass);
  s.loc = reinterpret_cast<int8_t*>(s.off + (1 << (k - L)));
  return s;
}

__device__ __forceinline__ uint32_t gidx(const TileShared& s, uint32_t base, uint32_t j, int L) {
  return base + (uint32_t)s.off[j >> L] + (j & ((1u << L) - 1u));
}

// Per-CTA set-up: offsets, local bits and this row's gate tensors (K0).
__device__ void setup(const SweepArgs& a, const TiledDev& t, const TileShared& s, int64_t b, int kk,
                      int* bad) {
  const int noff = 1 << (t.k - t.L);
  for (int i = threadIdx.x; i < noff; i += blockDim.x) s.off[i] = t.off[i];
  if (threadIdx.x < 32) s.loc[threadIdx.x] = t.loc[threadIdx.x];
  // shifted gates are numbered in pass order (tiled_compile)
  for (int i = threadIdx.x; i < t.nrec; i += blockDim.x) {
    s.mats[i] = build_recipe(a, t.ops, t.rec_ptr, t.rec_ops, t.rec0 + i, b, kk, bad);
    s.gpart[3 * i] = s.gpart[3 * i + 1] = s.gpart[3 * i + 2] = 0.0;
  }
  for (int i = threadIdx.x; i < t.ndops; i += blockDim.x) s.dops[i] = t.dops[i];
  for (int g = threadIdx.x; g < a.n_groups; g += blockDim.x) s.vsum[g] = 0.0;
  __syncthreads();
}

__device__ void flush_grads(const SweepArgs& a, const TiledDev& t, const TileShared& s, int lr) {
  __syncthreads();
  for (int i = t.bo0 + (int)threadIdx.x; i < t.bo1; i += blockDim.x) {
    const DOp d = s.dops[i];
    for (int j = 0; j < d.nang; j++)
      if (d.slot[j] >= 0) atomicAdd(&t.gacc[(int64_t)lr * a.P + d.slot[j]], s.gpart[3 * d.mat + j]);
  }
}

__device__ void forward_tile(const TiledDev& t, const TileShared& s, const TileCtx& ctx) {
  const int ngroups = 1 << (t.k - kFwdRegBits);
  for (int i = 0; i < t.nfp; i++) {
    const RegPass rp = t.fp[i];
    for (int grp = threadIdx.x; grp < ngroups; grp += blockDim.x)
      fwd_group<kFwdRegBits>(s.psi, rp, s.dops, s.mats, ctx.base, (uint32_t)grp);
    __syncthreads();
  }
}

__device__ void reverse_tile(const TiledDev& t, const TileShared& s, const TileCtx& ctx) {
  const int ngroups = 1 << (t.k - kRevRegBits);
  for (int i = t.nbp - 1; i >= 0; i--) {
    const RegPass rp = t.bp[i];
    for (int g0 = 0; g0 < ngroups; g0 += blockDim.x)
      adj_group<kRevRegBits, false>(s.psi, s.lam, rp, s.dops, s.mats, ctx.base, (uint32_t)(g0 + threadIdx.x),
                          g0 + (int)threadIdx.x < ngroups, s.gpart);
    __syncthreads();
  }
}

// Forward pass.  FIRST: the tile starts as |0...0> instead of being read.
// LAST: accumulate the observable groups; with GRAD also form lambda = O_w psi
// and run this pass's reverse sweep at once (psi and lambda then written).
template <bool FIRST, bool LAST, bool GRAD>
__global__ void __launch_bounds__(256) k1_forward(SweepArgs a, TiledDev t, int store) {
  extern __shared__ __align__(16) unsigned char raw[];
  const TileShared s = carve(raw, t.k, t.L, GRAD && LAST, t.nrec, t.ndops, a.n_groups);
  const int lr = blockIdx.y;
  const int row = t.row0 + lr;
  const int64_t b = row / a.ps_copies;
  const int kk = row % a.ps_copies;
  int bad = 0;
  setup(a, t, s, b, kk, &bad);
  if (bad) atomicOr(a.status, 1 << TDQ_ERR_NONFINITE);
  const uint32_t nloc = 1u << t.k;
  const uint32_t dim = 1u << t.n;
  c2* gpsi = t.psi + (size_t)lr * dim;
  c2* glam = GRAD ? t.lam + (size_t)lr * dim : nullptr;
  const uint32_t other = (dim - 1u) & ~t.smask;
  const int tile0 = blockIdx.x * t.tiles_per_cta;
  const int tile1 = min(t.ntiles, tile0 + t.tiles_per_cta);
  for (int tile = tile0; tile < tile1; tile++) {
    const uint32_t base = deposit((uint32_t)tile, other);
    if (FIRST) {
      for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x)
        s.psi[swz(j)] = {(base == 0u && j == 0u) ? 1.f : 0.f, 0.f};
    } else {
      for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) s.psi[swz(j)] = gpsi[gidx(s, base, j, t.L)];
    }
    __syncthreads();
    const TileCtx ctx{s.loc, base, t.k};
    forward_tile(t, s, ctx);
    if (LAST && a.output == TDQ_OUT_EXPVAL) {
      for (int g = 0; g < a.n_groups; g++) {
        float acc = 0.f;
        for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) {
          const c2 v = s.psi[swz(j)];
          acc += (v.x * v.x + v.y * v.y) *
                 diag_weight(a.terms, a.group_ptr[g], a.group_ptr[g + 1], gidx(s, base, j, t.L));
        }
        acc = warp_sum_f(acc);
        if ((threadIdx.x & 31) == 0) atomicAdd(&s.vsum[g], (double)acc);
      }
      if (GRAD) {
        for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) {
          const uint32_t x = gidx(s, base, j, t.L);
          float d = 0.f;
          for (int g = 0; g < a.n_groups; g++) {
            const float w = a.gw ? (float)a.gw[b * a.n_groups + g] : 1.f;
            d += w * diag_weight(a.terms, a.group_ptr[g], a.group_ptr[g + 1], x);
          }
          const c2 v = s.psi[swz(j)];
          s.lam[swz(j)] = {d * v.x, d * v.y};
        }
        __syncthreads();
        reverse_tile(t, s, ctx);
        for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) {
          const uint32_t x = gidx(s, base, j, t.L);
          gpsi[x] = s.psi[swz(j)];
          glam[x] = s.lam[swz(j)];
        }
      }
    }
    if (!(LAST && GRAD) && store) {
      for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) gpsi[gidx(s, base, j, t.L)] = s.psi[swz(j)];
    }
    __syncthreads();
  }
  if (LAST && a.output == TDQ_OUT_EXPVAL) {
    __syncthreads();
    for (int g = threadIdx.x; g < a.n_groups; g += blockDim.x)
      atomicAdd(&t.vals[(int64_t)lr * a.n_groups + g], s.vsum[g]);
  }
  if (GRAD && LAST) flush_grads(a, t, s, lr);
}

// Reverse pass over the tiles of one pass (passes before the last).
__global__ void __launch_bounds__(256) k1_reverse(SweepArgs a, TiledDev t) {
  extern __shared__ __align__(16) unsigned char raw[];
  const TileShared s = carve(raw, t.k, t.L, true, t.nrec, t.ndops, a.n_groups);
  const int lr = blockIdx.y;
  const int row = t.row0 + lr;
  const int64_t b = row / a.ps_copies;
  int bad = 0;
  setup(a, t, s, b, 0, &bad);
  const uint32_t nloc = 1u << t.k;
  const uint32_t dim = 1u << t.n;
  c2* gpsi = t.psi + (size_t)lr * dim;
  c2* glam = t.lam + (size_t)lr * dim;
  const uint32_t other = (dim - 1u) & ~t.smask;
  const int tile0 = blockIdx.x * t.tiles_per_cta;
  const int tile1 = min(t.ntiles, tile0 + t.tiles_per_cta);
  for (int tile = tile0; tile < tile1; tile++) {
    const uint32_t base = deposit((uint32_t)tile, other);
    for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) {
      const uint32_t x = gidx(s, base, j, t.L);
      s.psi[swz(j)] = gpsi[x];
      s.lam[swz(j)] = glam[x];
    }
    __syncthreads();
    const TileCtx ctx{s.loc, base, t.k};
    reverse_tile(t, s, ctx);
    for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) {
      const uint32_t x = gidx(s, base, j, t.L);
      gpsi[x] = s.psi[swz(j)];
      glam[x] = s.lam[swz(j)];
    }
    __syncthreads();
  }
  flush_grads(a, t, s, lr);
}

// Copy out the chunk's values, F for the shift rule, gradients, amplitudes.
__global__ void k1_finalize(SweepArgs a, TiledDev t, int nrows, int grad_adj) {
  const int lr = blockIdx.x;
  if (lr >= nrows) return;
  const int row = t.row0 + lr;
  const int64_t b = row / a.ps_copies;
  const int kk = row % a.ps_copies;
  if (a.output == TDQ_OUT_EXPVAL) {
    if (threadIdx.x == 0) {
      double F = 0.0;
      for (int g = 0; g < a.n_groups; g++) {
        const double v = t.vals[(int64_t)lr * a.n_groups + g];
        F += (a.gw ? a.gw[b * a.n_groups + g] : 1.0) * v;
        if (kk == 0) a.values[b * a.n_groups + g] = v;
      }
      if (a.ps_copies > 1) a.ps_F[row] = F;
    }
  } else if (kk == 0) {
    const c2* psi = t.psi + (size_t)lr * (1u << t.n);
    for (int i = threadIdx.x; i < a.A; i += blockDim.x) {
      const c2 v = psi[a.amp_idx[i]];
      a.values[(b * a.A + i) * 2] = v.x;
      a.values[(b * a.A + i) * 2 + 1] = v.y;
    }
  }
  if (grad_adj)
    for (int j = threadIdx.x; j < a.P; j += blockDim.x) a.grads[b * a.P + j] = (float)t.gacc[(int64_t)lr * a.P + j];
}

size_t smem_for(int k, int L, bool two, int nrec, int ndops, int ng) {
  return (size_t)(1 << k) * sizeof(c2) * (two ? 2 : 1) + sizeof(OpMat) * nrec + sizeof(DOp) * ndops +
         (32 + (size_t)ng) * sizeof(double) + 3 * sizeof(double) * nrec + sizeof(int) * (1 << (k - L)) +
         32 + 16;
}

}  // namespace

void tiled_free(TiledSweep& t) {
  cudaFree(t.d_ops);
  cudaFree(t.d_off);
  cudaFree(t.d_loc);
  cudaFree(t.d_psi);
  cudaFree(t.d_lam);
  cudaFree(t.d_gacc);
  cudaFree(t.d_vals);
  cudaFree(t.d_ps_gate_pass);
  cudaFree(t.d_rpass);
  cudaFree(t.d_dops);
  cudaFree(t.d_rec_ptr);
  cudaFree(t.d_rec_ops);
  t.d_ps_gate_pass = nullptr;
  t.d_rpass = nullptr;
  t.d_dops = nullptr;
  t.d_rec_ptr = t.d_rec_ops = nullptr;
  t.d_ops = nullptr;
  t.d_off = nullptr;
  t.d_loc = nullptr;
  t.d_psi = t.d_lam = nullptr;
  t.d_gacc = t.d_vals = nullptr;
}

// Needs a gate on bit position p held in the tile?  (diagonal gates never,
// CNOT only for its target)
static void tile_needs(const SweepOp& op, std::vector<int>& need) {
  need.clear();
  switch (op.kind) {
    case K_RZ: case K_Z: case K_CZ: case K_RZZ: break;
    case K_CNOT: need.push_back(op.p1); break;
    default: need.push_back(op.p0); break;
  }
}

tdq_status tiled_compile(TiledSweep& t, const tdq_circuit* c, const std::vector<SweepOp>& ops,
                         const std::vector<int>& ps_gate, int rows, bool adj, int tile_qubits,
                         double* bytes_row) {
  const int n = c->n;
  t.n = n;
  const int kq = tile_qubits > 0 ? tile_qubits : 12;
  if (kq < 5 || kq > 13) return fail(TDQ_ERR_ARG, "tile_qubits must be in 5..13");
  t.k = std::min(n, kq);
  t.L = std::min(4, t.k);
  t.adj = adj;
  t.rows = rows;
  t.P = c->n_params;
  t.ng = c->n_groups;
  if (t.ng > 1024) return fail(TDQ_ERR_UNSUPPORTED, "tiled sweep: more than 1024 output groups");
  const int G = (int)ops.size();
  // Greedy pass schedule: walk gates in circuit order; take a gate when every
  // earlier gate on its qubits is taken and its non-diagonal bits fit in the
  // tile (growing the tile's bit set up to k); otherwise block its qubits for
  // the rest of this pass.
  std::vector<char> done(G, 0);
  std::vector<int> order;
  int remaining = G, first = 0;
  t.passes.clear();
  std::vector<int> need;
  while (remaining > 0) {
    uint32_t smask = (1u << t.L) - 1u;
    int used = t.L;
    std::vector<char> blocked(n, 0);
    TiledPass ps{0, (int)order.size(), 0};
    while (first < G && done[first]) first++;
    for (int g = first; g < G; g++) {
      if (done[g]) continue;
      const SweepOp& op = ops[g];
      const int pa = op.p0, pb = op.p1;
      if (blocked[pa] || (pb >= 0 && blocked[pb])) {
        blocked[pa] = 1;
        if (pb >= 0) blocked[pb] = 1;
        continue;
      }
      tile_needs(op, need);
      uint32_t add = 0;
      for (int p : need)
        if (!((smask >> p) & 1u)) add |= 1u << p;
      if (used + __builtin_popcount(add) <= t.k) {
        smask |= add;
        used += __builtin_popcount(add);
        done[g] = 1;
        remaining--;
        order.push_back(g);
      } else {
        blocked[pa] = 1;
        if (pb >= 0) blocked[pb] = 1;
      }
    }
    // fill the tile's unused slots with the lowest free positions
    for (int p = 0; p < n && used < t.k; p++)
      if (!((smask >> p) & 1u)) {
        smask |= 1u << p;
        used++;
      }
    ps.smask = smask;
    ps.op_end = (int)order.size();
    if (ps.op_end == ps.op_begin) return fail(TDQ_ERR_STATE, "tiled sweep: empty pass");
    t.passes.push_back(ps);
  }
  // device program in pass order; slot/src stay per op
  std::vector<SweepOp> pops;
  for (int g : order) pops.push_back(ops[g]);
  std::vector<int> offs;
  std::vector<int8_t> locs;
  int maxp = 0;
  for (const TiledPass& ps : t.passes) {
    maxp = std::max(maxp, ps.op_end - ps.op_begin);
    std::vector<int> hi;
    int8_t loc[32];
    for (int p = 0; p < 32; p++) loc[p] = -1;
    int li = 0;
    for (int p = 0; p < n; p++)
      if ((ps.smask >> p) & 1u) {
        loc[p] = (int8_t)li++;
        if (p >= t.L) hi.push_back(p);
      }
    const int nh = t.k - t.L;
    for (int j = 0; j < (1 << nh); j++) {
      int o = 0;
      for (int i = 0; i < nh; i++)
        if ((j >> i) & 1) o |= 1 << hi[i];
      offs.push_back(o);
    }
    for (int p = 0; p < 32; p++) locs.push_back(loc[p]);
  }
  // decoded programs inside every tile pass (op indices are pass-ordered):
  // a fused forward program and, with gradients, a one-op-per-gate reverse one
  Program prog;
  t.max_rec = 0;
  int max_dops = 0;
  for (size_t pi = 0; pi < t.passes.size(); pi++) {
    const int r0 = (int)prog.rec_ptr.size() - 1, d0 = (int)prog.dops.size();
    t.rec_begin.push_back(r0);
    t.fp_begin.push_back((int)prog.passes.size());
    build_program(pops, t.passes[pi].op_begin, t.passes[pi].op_end, &locs[pi * 32], t.k, true, r0, kFwdRegBits, prog);
    t.fp_end.push_back((int)prog.passes.size());
    const int bd0 = (int)prog.dops.size();
    t.bp_begin.push_back((int)prog.passes.size());
    if (adj) build_program(pops, t.passes[pi].op_begin, t.passes[pi].op_end, &locs[pi * 32], t.k, false, r0, kRevRegBits, prog);
    t.bp_end.push_back((int)prog.passes.size());
    t.bo_begin.push_back(bd0 - d0);
    t.bo_end.push_back((int)prog.dops.size() - d0);
    t.rec_end.push_back((int)prog.rec_ptr.size() - 1);
    for (int q = t.fp_begin.back(); q < t.bp_end.back(); q++) {  // op ranges relative to the tile pass
      prog.passes[q].op_begin -= d0;
      prog.passes[q].op_end -= d0;
    }
    t.dop_begin.push_back(d0);
    t.dop_end.push_back((int)prog.dops.size());
    t.max_rec = std::max(t.max_rec, t.rec_end.back() - r0);
    max_dops = std::max(max_dops, (int)prog.dops.size() - d0);
  }
  t.max_dops = max_dops;
  t.max_pass_ops = maxp;
  // parameter-shift copies refer to gates by index: renumber to pass order
  t.order = order;
  std::vector<int> pos(G, 0), psp;
  for (int i = 0; i < G; i++) pos[order[i]] = i;
  for (int g : ps_gate) psp.push_back(pos[g]);
  auto up = [](void** d, const void* h, size_t bytes) -> tdq_status {
    if (cudaMalloc(d, bytes) != cudaSuccess) return fail(TDQ_ERR_OOM, "tiled sweep: cudaMalloc");
    if (cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(TDQ_ERR_CUDA, "tiled sweep: cudaMemcpy");
    return TDQ_OK;
  };
  tdq_status s;
  if ((s = up((void**)&t.d_ops, pops.data(), sizeof(SweepOp) * pops.size())) != TDQ_OK) return s;
  if ((s = up((void**)&t.d_off, offs.data(), sizeof(int) * offs.size())) != TDQ_OK) return s;
  if ((s = up((void**)&t.d_loc, locs.data(), locs.size())) != TDQ_OK) return s;
  if (!psp.empty() && (s = up((void**)&t.d_ps_gate_pass, psp.data(), sizeof(int) * psp.size())) != TDQ_OK)
    return s;
  if ((s = up((void**)&t.d_rpass, prog.passes.data(), sizeof(RegPass) * prog.passes.size())) != TDQ_OK) return s;
  if ((s = up((void**)&t.d_dops, prog.dops.data(), sizeof(DOp) * prog.dops.size())) != TDQ_OK) return s;
  if ((s = up((void**)&t.d_rec_ptr, prog.rec_ptr.data(), sizeof(int) * prog.rec_ptr.size())) != TDQ_OK) return s;
  if ((s = up((void**)&t.d_rec_ops, prog.rec_ops.data(), sizeof(int) * prog.rec_ops.size())) != TDQ_OK) return s;
  // resident rows: bounded by a workspace budget of 3/4 of free memory, 64 GiB at most
  size_t freeb = 0, totb = 0;
  cudaMemGetInfo(&freeb, &totb);
  const size_t per_row = ((size_t)1 << n) * sizeof(c2) * (adj ? 2 : 1);
  size_t budget = std::min<size_t>((size_t)64 << 30, freeb / 4 * 3);
  t.chunk_rows = (int)std::max<size_t>(1, std::min<size_t>((size_t)rows, budget / per_row));
  if ((size_t)t.chunk_rows * per_row > freeb) return fail(TDQ_ERR_OOM, "tiled sweep: state does not fit");
  if (cudaMalloc(&t.d_psi, ((size_t)1 << n) * sizeof(c2) * t.chunk_rows) != cudaSuccess)
    return fail(TDQ_ERR_OOM, "tiled sweep: state buffer");
  if (adj && cudaMalloc(&t.d_lam, ((size_t)1 << n) * sizeof(c2) * t.chunk_rows) != cudaSuccess)
    return fail(TDQ_ERR_OOM, "tiled sweep: adjoint buffer");
  if (cudaMalloc(&t.d_gacc, sizeof(double) * std::max(1, t.P) * t.chunk_rows) != cudaSuccess)
    return fail(TDQ_ERR_OOM, "tiled sweep: gradient buffer");
  if (cudaMalloc(&t.d_vals, sizeof(double) * std::max(1, t.ng) * t.chunk_rows) != cudaSuccess)
    return fail(TDQ_ERR_OOM, "tiled sweep: value buffer");
  const size_t sm_fwd = smem_for(t.k, t.L, adj, t.max_rec, t.max_dops, t.ng);
  if (sm_fwd > 227 * 1024) return fail(TDQ_ERR_UNSUPPORTED, "tiled sweep: tile program too large");
  cudaFuncSetAttribute(k1_forward<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fwd);
  cudaFuncSetAttribute(k1_forward<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fwd);
  cudaFuncSetAttribute(k1_forward<true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fwd);
  cudaFuncSetAttribute(k1_forward<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fwd);
  cudaFuncSetAttribute(k1_forward<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fwd);
  cudaFuncSetAttribute(k1_forward<false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fwd);
  cudaFuncSetAttribute(k1_reverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fwd);
  // HBM traffic model per row: every pass reads and writes the state (the
  // first pass only writes it, a value-only last pass only reads it); with the
  // reverse sweep each earlier pass reads and writes psi and lambda again.
  const double sb = (double)((size_t)1 << n) * sizeof(c2);
  const int np = (int)t.passes.size();
  double by = 0;
  for (int p = 0; p < np; p++) {
    const bool f = p == 0, l = p == np - 1;
    by += (f ? 0 : sb) + ((l && !adj && c->n_groups > 0) ? 0 : sb);
    if (adj && l) by += sb;  // lambda written by the fused last pass
    if (adj && !l) by += 4 * sb;
  }
  *bytes_row = by;
  return TDQ_OK;
}

static void set_pass(const TiledSweep& t, TiledDev& d, int p) {
  d.fp = t.d_rpass + t.fp_begin[p];
  d.nfp = t.fp_end[p] - t.fp_begin[p];
  d.bp = t.d_rpass + t.bp_begin[p];
  d.nbp = t.bp_end[p] - t.bp_begin[p];
  d.dops = t.d_dops + t.dop_begin[p];
  d.ndops = t.dop_end[p] - t.dop_begin[p];
  d.bo0 = t.bo_begin[p];
  d.bo1 = t.bo_end[p];
  d.rec_ptr = t.d_rec_ptr;
  d.rec_ops = t.d_rec_ops;
  d.rec0 = t.rec_begin[p];
  d.nrec = t.rec_end[p] - t.rec_begin[p];
}

tdq_status tiled_execute(TiledSweep& t, const SweepArgs& a0, int grad, cudaStream_t st,
                         int* launches) {
  SweepArgs a = a0;
  if (a.ps_copies > 1) a.ps_gate = t.d_ps_gate_pass;
  const bool adj = grad == TDQ_GRAD_ADJOINT;
  const int np = (int)t.passes.size();
  const int ntiles = 1 << (t.n - t.k);
  const size_t sm = smem_for(t.k, t.L, adj, t.max_rec, t.max_dops, t.ng);
  for (int row0 = 0; row0 < t.rows; row0 += t.chunk_rows) {
    const int nr = std::min(t.chunk_rows, t.rows - row0);
    if (cudaMemsetAsync(t.d_vals, 0, sizeof(double) * std::max(1, t.ng) * nr, st) != cudaSuccess)
      return fail(TDQ_ERR_CUDA, "tiled sweep: memset");
    if (adj && cudaMemsetAsync(t.d_gacc, 0, sizeof(double) * std::max(1, t.P) * nr, st) != cudaSuccess)
      return fail(TDQ_ERR_CUDA, "tiled sweep: memset");
    // CTAs per row: enough CTAs for ~4 per SM over the chunk
    const int want = std::max(1, (152 * 4 + nr - 1) / nr);
    const int cpr = std::min(ntiles, want);
    const int tpc = (ntiles + cpr - 1) / cpr;
    const int cpr2 = (ntiles + tpc - 1) / tpc;
    const dim3 grid(cpr2, nr);
    TiledDev d{};
    d.ops = t.d_ops;
    d.psi = t.d_psi;
    d.lam = t.d_lam;
    d.gacc = t.d_gacc;
    d.vals = t.d_vals;
    d.n = t.n;
    d.k = t.k;
    d.L = t.L;
    d.tiles_per_cta = tpc;
    d.ntiles = ntiles;
    d.row0 = row0;
    const int nthr = std::max(32, std::min(256, 1 << (t.k - kFwdRegBits)));
    const int store_last = (a.output == TDQ_OUT_AMPLITUDE) ? 1 : 0;
    for (int p = 0; p < np; p++) {
      d.off = t.d_off + (size_t)p * (1 << (t.k - t.L));
      d.loc = t.d_loc + (size_t)p * 32;
      d.smask = t.passes[p].smask;
      d.op_begin = t.passes[p].op_begin;
      d.op_end = t.passes[p].op_end;
      set_pass(t, d, p);
      const bool f = p == 0, l = p == np - 1;
      if (f && !l) k1_forward<true, false, false><<<grid, nthr, sm, st>>>(a, d, 1);
      else if (!f && !l) k1_forward<false, false, false><<<grid, nthr, sm, st>>>(a, d, 1);
      else if (f && l && !adj) k1_forward<true, true, false><<<grid, nthr, sm, st>>>(a, d, store_last);
      else if (!f && l && !adj) k1_forward<false, true, false><<<grid, nthr, sm, st>>>(a, d, store_last);
      else if (f && l && adj) k1_forward<true, true, true><<<grid, nthr, sm, st>>>(a, d, 1);
      else k1_forward<false, true, true><<<grid, nthr, sm, st>>>(a, d, 1);
      (*launches)++;
    }
    if (adj) {
      for (int p = np - 2; p >= 0; p--) {
        d.off = t.d_off + (size_t)p * (1 << (t.k - t.L));
        d.loc = t.d_loc + (size_t)p * 32;
        d.smask = t.passes[p].smask;
        d.op_begin = t.passes[p].op_begin;
        d.op_end = t.passes[p].op_end;
        set_pass(t, d, p);
        k1_reverse<<<grid, nthr, sm, st>>>(a, d);
        (*launches)++;
      }
    }
    k1_finalize<<<nr, 128, 0, st>>>(a, d, nr, adj ? 1 : 0);
    (*launches)++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TDQ_ERR_CUDA, std::string("tiled sweep launch: ") + cudaGetErrorString(e));
  }
  return TDQ_OK;
}

}  // namespace tdq
