// Kernel K1: tiled state sweep through HBM (see sweep_tiled.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "k1_body.cuh"
#include "sweep_jit.h"
#include "sweep_tiled.cuh"

namespace tdq {

namespace {

template <bool FIRST, bool LAST, bool GRAD>
__global__ void __launch_bounds__(256) k1_forward(SweepArgs a, TiledDev t, int store) {
  k1_forward_body<FIRST, LAST, GRAD, InterpTile>(a, t, store);
}

__global__ void __launch_bounds__(256) k1_reverse(SweepArgs a, TiledDev t) { k1_reverse_body<InterpTile>(a, t); }

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
  } else if (kk == 0 && a.output == TDQ_OUT_AMPLITUDE) {
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

// The chunk's final states as the output: the whole state (TDQ_OUT_STATE) or
// the probabilities (TDQ_OUT_PROBS) of every row, grid-stride over (row, x).
__global__ void k1_state_out(SweepArgs a, TiledDev t, int nrows) {
  const int64_t dim = (int64_t)1 << t.n, tot = dim * nrows;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int lr = (int)(i / dim);
    const int row = t.row0 + lr;
    if (row % a.ps_copies) continue;
    const int64_t b = row / a.ps_copies, x = i - (int64_t)lr * dim;
    const c2 v = t.psi[i];
    if (a.output == TDQ_OUT_STATE) {
      a.values[(b * dim + x) * 2] = v.x;
      a.values[(b * dim + x) * 2 + 1] = v.y;
    } else {
      a.values[b * dim + x] = (double)v.x * v.x + (double)v.y * v.y;
    }
  }
}

}  // namespace

void tiled_free(TiledSweep& t) {
  for (cudaEvent_t e : t.ev) cudaEventDestroy(e);
  t.ev.clear();
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

tdq_status tiled_plan(TiledSweep& t, const tdq_circuit* c, const std::vector<SweepOp>& ops,
                      const std::vector<int>& ps_gate, int rows, bool adj, int tile_qubits, int fb, int rb,
                      TiledHost& h) {
  t.fb = fb;
  t.rb = rb;
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
  std::vector<SweepOp>& pops = h.pops;
  for (int g : order) pops.push_back(ops[g]);
  std::vector<int>& offs = h.offs;
  std::vector<int8_t>& locs = h.locs;
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
  Program& prog = h.prog;
  t.max_rec = 0;
  int max_dops = 0;
  for (size_t pi = 0; pi < t.passes.size(); pi++) {
    const int r0 = (int)prog.rec_ptr.size() - 1, d0 = (int)prog.dops.size();
    t.rec_begin.push_back(r0);
    t.fp_begin.push_back((int)prog.passes.size());
    build_program(pops, t.passes[pi].op_begin, t.passes[pi].op_end, &locs[pi * 32], t.k, true, r0, fb, prog);
    t.fp_end.push_back((int)prog.passes.size());
    const int bd0 = (int)prog.dops.size();
    t.bp_begin.push_back((int)prog.passes.size());
    if (adj) build_program(pops, t.passes[pi].op_begin, t.passes[pi].op_end, &locs[pi * 32], t.k, false, r0, rb, prog);
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
  std::vector<int> pos(G, 0);
  std::vector<int>& psp = h.psp;
  for (int i = 0; i < G; i++) pos[order[i]] = i;
  for (int g : ps_gate) psp.push_back(pos[g]);
  return TDQ_OK;
}

tdq_status tiled_compile(TiledSweep& t, const tdq_circuit* c, const std::vector<SweepOp>& ops,
                         const std::vector<int>& ps_gate, int rows, bool adj, int tile_qubits, bool interpret,
                         int fb, int rb, double* bytes_row) {
  TiledHost h;
  tdq_status s0 = tiled_plan(t, c, ops, ps_gate, rows, adj, tile_qubits, fb, rb, h);
  if (s0 != TDQ_OK) return s0;
  const int n = c->n;
  const std::vector<SweepOp>& pops = h.pops;
  const std::vector<int>& offs = h.offs;
  const std::vector<int8_t>& locs = h.locs;
  const Program& prog = h.prog;
  const std::vector<int>& psp = h.psp;
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
  // threads: one forward group (2^4 amplitudes) per thread; reverse kernels
  // up to 256 threads (two CTAs per SM)
  t.nthreads = std::max(32, std::min(256, 1 << (t.k - fb)));
  t.nthreads_r = interpret ? t.nthreads : std::max(32, std::min(256, 1 << (t.k - rb)));
  t.kf.clear();
  t.kr.clear();
  t.spec_gbytes.clear();
  const int np = (int)t.passes.size();
  int gmax = 0, ndops_sm = 0;
  std::string src;
  if (!interpret) {
    // every tile pass as straight-line code; one compilation for all passes
    std::vector<int> nacc;
    src = k1_specialised_source(t, prog, t.nthreads, t.nthreads_r, &nacc);
    const int nw = std::max(t.nthreads, t.nthreads_r) / 32;
    for (int p = 0; p < np; p++) {
      t.spec_gbytes.push_back(4 * nw * std::max(1, nacc[p]));
      gmax = std::max(gmax, t.spec_gbytes.back());
    }
  } else {
    gmax = 24 * t.max_rec;
    ndops_sm = t.max_dops;
  }
  // shared memory per kernel: forward kernels a double-buffered state (psi;
  // the last pass also lambda; one buffer where two do not fit).  Reverse
  // kernels hold psi and lambda in one buffer each: two CTAs of 256 threads
  // per SM then interleave one CTA's tile loads with the other's compute,
  // which measured faster than one double-buffered CTA of 512 threads.
  auto sizes = [&](int nb) {
    t.smem_f.assign(np, 0);
    for (int p = 0; p < np; p++)
      t.smem_f[p] = k1_smem_bytes(t.k, t.L, p == 0 ? 1 : nb, (adj && p == np - 1) ? 1 : 0, t.max_rec, ndops_sm,
                                  t.ng, gmax);
    t.smem_r = adj ? k1_smem_bytes(t.k, t.L, 1, 1, t.max_rec, ndops_sm, t.ng, gmax) : 0;
    size_t m = t.smem_r;
    for (size_t v : t.smem_f) m = std::max(m, v);
    return m;
  };
  t.dbl = sizes(2) <= 227 * 1024 ? 1 : 0;
  size_t smax = sizes(t.dbl ? 2 : 1);
  if (smax > 227 * 1024) return fail(TDQ_ERR_UNSUPPORTED, "tiled sweep: tile program too large");
  if (!interpret) {
    for (int p = 0; p < np; p++) {
      const void* kf = nullptr;
      const void* kr = nullptr;
      const std::string nf = "tdq_k1f_" + std::to_string(p), nr = "tdq_k1r_" + std::to_string(p);
      tdq_status s2 = jit_kernel(src, nf.c_str(), &kf);
      if (s2 != TDQ_OK) return s2;
      if (cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.smem_f[p]) != cudaSuccess)
        return fail(TDQ_ERR_CUDA, "tiled sweep: cudaFuncSetAttribute");
      if (adj && p + 1 < np) {
        if ((s2 = jit_kernel(src, nr.c_str(), &kr)) != TDQ_OK) return s2;
        if (cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.smem_r) != cudaSuccess)
          return fail(TDQ_ERR_CUDA, "tiled sweep: cudaFuncSetAttribute");
      }
      t.kf.push_back(kf);
      t.kr.push_back(kr);
    }
  } else {
    const int sm = (int)smax;
    cudaFuncSetAttribute(k1_forward<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k1_forward<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k1_forward<true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k1_forward<false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k1_forward<true, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k1_forward<false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k1_reverse, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  }
  // resident CTAs per kernel (occupancy of the kernel at its launch shape)
  {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    auto slots = [&](const void* fn, int threads, size_t smem) {
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
      }
      return std::max(1, nsm) * nb;
    };
    t.slots_f.assign(np, 0);
    for (int p = 0; p < np; p++) {
      const bool f = p == 0, l = p == np - 1;
      const void* fn = !t.kf.empty() ? t.kf[p]
                       : (f && !l) ? (const void*)k1_forward<true, false, false>
                       : (!f && !l) ? (const void*)k1_forward<false, false, false>
                       : (f && !adj) ? (const void*)k1_forward<true, true, false>
                       : (!adj) ? (const void*)k1_forward<false, true, false>
                       : f ? (const void*)k1_forward<true, true, true>
                           : (const void*)k1_forward<false, true, true>;
      t.slots_f[p] = slots(fn, t.nthreads, t.smem_f[p]);
    }
    t.slots_r = nsm;
    if (adj && np > 1) t.slots_r = slots(!t.kr.empty() ? t.kr[0] : (const void*)k1_reverse, t.nthreads_r, t.smem_r);
  }
  // HBM traffic model per row: every pass reads and writes the state (the
  // first pass only writes it, a value-only last pass only reads it); with the
  // reverse sweep each earlier pass reads and writes psi and lambda again.
  const double sb = (double)((size_t)1 << n) * sizeof(c2);
  double by = 0;
  for (int p = 0; p < np; p++) {
    const bool f = p == 0, l = p == np - 1;
    by += (f ? 0 : sb) + ((l && !adj && c->n_groups > 0) ? 0 : sb);
    if (adj && l) by += sb;  // lambda written by the fused last pass
    if (adj && !l) by += 4 * sb;
  }
  *bytes_row = by;
  // the same model per launch unit, with the algorithmic FLOPs of each pass
  // (forward passes, then the reverse passes from the second last down)
  const double dim = std::ldexp(1.0, n);
  const double obs = c->n_groups > 0 ? (3.0 + 2.0 * (double)c->terms.size()) * dim : 0.0;
  std::vector<double> fw(np, 0.0), dots(np, 0.0);
  for (int p = 0; p < np; p++)
    for (int o = t.passes[p].op_begin; o < t.passes[p].op_end; o++) {
      fw[p] += gate_fwd_flops(pops[o].kind, dim);
      dots[p] += gate_dot_flops(pops[o].kind, dim);
    }
  t.unit_flops.clear();
  t.unit_bytes.clear();
  t.unit_kind.clear();
  for (int p = 0; p < np; p++) {
    const bool f = p == 0, l = p == np - 1;
    t.unit_kind.push_back(l && adj ? 1 : 0);
    t.unit_flops.push_back(fw[p] + (l ? obs : 0.0) + (l && adj ? 2 * fw[p] + dots[p] + obs : 0.0));
    t.unit_bytes.push_back((f ? 0 : sb) + ((l && !adj && c->n_groups > 0) ? 0 : sb) + (adj && l ? sb : 0));
  }
  if (adj)
    for (int p = np - 2; p >= 0; p--) {
      t.unit_kind.push_back(2);
      t.unit_flops.push_back(2 * fw[p] + dots[p]);
      t.unit_bytes.push_back(4 * sb);
    }
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
  if (t.kf.empty()) {
    d.gbytes = 24 * d.nrec;
  } else {  // specialised: no decoded ops in shared memory; per-warp FP32 rows
    d.ndops = 0;
    d.gbytes = t.spec_gbytes[p];
  }
}

tdq_status tiled_execute(TiledSweep& t, const SweepArgs& a0, int grad, cudaStream_t st,
                         int* launches) {
  SweepArgs a = a0;
  if (a.ps_copies > 1) a.ps_gate = t.d_ps_gate_pass;
  const bool adj = grad == TDQ_GRAD_ADJOINT;
  const int np = (int)t.passes.size();
  const int ntiles = 1 << (t.n - t.k);
  for (int row0 = 0; row0 < t.rows; row0 += t.chunk_rows) {
    const int nr = std::min(t.chunk_rows, t.rows - row0);
    if (cudaMemsetAsync(t.d_vals, 0, sizeof(double) * std::max(1, t.ng) * nr, st) != cudaSuccess)
      return fail(TDQ_ERR_CUDA, "tiled sweep: memset");
    if (adj && cudaMemsetAsync(t.d_gacc, 0, sizeof(double) * std::max(1, t.P) * nr, st) != cudaSuccess)
      return fail(TDQ_ERR_CUDA, "tiled sweep: memset");
    // one wave per kernel: as many CTAs as fit on the GPU at once, each
    // with an equal share of the chunk's (row, tile) units
    const int64_t total = (int64_t)nr * ntiles;
    auto grid_for = [&](int slots, TiledDev& dd) {
      const int64_t n0 = std::max<int64_t>(1, std::min<int64_t>(total, slots));
      const int64_t upc = (total + n0 - 1) / n0;
      dd.tiles_per_cta = (int)upc;
      return dim3((unsigned)((total + upc - 1) / upc));
    };
    TiledDev d{};
    d.ops = t.d_ops;
    d.psi = t.d_psi;
    d.lam = t.d_lam;
    d.gacc = t.d_gacc;
    d.vals = t.d_vals;
    d.n = t.n;
    d.k = t.k;
    d.L = t.L;
    d.ntiles = ntiles;
    d.row0 = row0;
    d.nrows = nr;
    d.dbl = t.dbl;
    const int nthr = t.nthreads;
    const int store_last = (a.output != TDQ_OUT_EXPVAL) ? 1 : 0;  // amplitudes, states: read from HBM
    for (int p = 0; p < np; p++) {
      d.off = t.d_off + (size_t)p * (1 << (t.k - t.L));
      d.loc = t.d_loc + (size_t)p * 32;
      d.smask = t.passes[p].smask;
      d.op_begin = t.passes[p].op_begin;
      d.op_end = t.passes[p].op_end;
      set_pass(t, d, p);
      const bool f = p == 0, l = p == np - 1;
      const dim3 grid = grid_for(t.slots_f[p], d);
      const bool rec = !t.ev.empty() && row0 == 0;
      if (rec) cudaEventRecord(t.ev[2 * p], st);
      if (!t.kf.empty()) {
        int st_flag = (l && !adj) ? store_last : 1;
        void* args[] = {&a, &d, &st_flag};
        if (cudaLaunchKernel(t.kf[p], grid, dim3(nthr), args, t.smem_f[p], st) != cudaSuccess)
          return fail(TDQ_ERR_CUDA, "tiled sweep: launch of a specialised pass");
        if (rec) cudaEventRecord(t.ev[2 * p + 1], st);
        (*launches)++;
        continue;
      }
      const size_t sm = t.smem_f[p];
      if (f && !l) k1_forward<true, false, false><<<grid, nthr, sm, st>>>(a, d, 1);
      else if (!f && !l) k1_forward<false, false, false><<<grid, nthr, sm, st>>>(a, d, 1);
      else if (f && l && !adj) k1_forward<true, true, false><<<grid, nthr, sm, st>>>(a, d, store_last);
      else if (!f && l && !adj) k1_forward<false, true, false><<<grid, nthr, sm, st>>>(a, d, store_last);
      else if (f && l && adj) k1_forward<true, true, true><<<grid, nthr, sm, st>>>(a, d, 1);
      else k1_forward<false, true, true><<<grid, nthr, sm, st>>>(a, d, 1);
      if (rec) cudaEventRecord(t.ev[2 * p + 1], st);
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
        const dim3 grid = grid_for(t.slots_r, d);
        d.dbl = 0;  // reverse kernels: one buffer per state (see tiled_compile)
        const int u = np + (np - 2 - p);  // launch unit of this reverse pass
        const bool rec = !t.ev.empty() && row0 == 0;
        if (rec) cudaEventRecord(t.ev[2 * u], st);
        if (!t.kr.empty()) {
          void* args[] = {&a, &d};
          if (cudaLaunchKernel(t.kr[p], grid, dim3(t.nthreads_r), args, t.smem_r, st) != cudaSuccess)
            return fail(TDQ_ERR_CUDA, "tiled sweep: launch of a specialised pass");
        } else {
          k1_reverse<<<grid, t.nthreads_r, t.smem_r, st>>>(a, d);
        }
        if (rec) cudaEventRecord(t.ev[2 * u + 1], st);
        (*launches)++;
      }
    }
    k1_finalize<<<nr, 128, 0, st>>>(a, d, nr, adj ? 1 : 0);
    (*launches)++;
    if (a.output == TDQ_OUT_STATE || a.output == TDQ_OUT_PROBS) {
      const int64_t tot = (int64_t)nr << t.n;
      k1_state_out<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 8192), 256, 0, st>>>(a, d, nr);
      (*launches)++;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TDQ_ERR_CUDA, std::string("tiled sweep launch: ") + cudaGetErrorString(e));
  }
  return TDQ_OK;
}

}  // namespace tdq
