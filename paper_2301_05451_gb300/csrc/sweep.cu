// State-sweep execution of a circuit's tensor network (Sec. 3.2 (e), with the
// gradient by the reverse sweep of Sec. 4.1 or the shift rule of Sec. 4.2).
//
// Kernel K2 (this file): one CTA per batch row holds the whole rank-n ket
// tensor psi (2^n complex64) in shared memory, absorbs every gate tensor in
// circuit order (gate tensors are built from the row's angles in-kernel: K0
// fused), closes the network with the Z-product observables (K6) and, for
// gradients, runs the reverse sweep (K7): lambda = O psi, then per gate g from
// last to first   psi <- G^dagger psi,  dF/da += 2 Re <lambda| dG/da |psi>,
// lambda <- G^dagger lambda   (psi is un-computed instead of stored).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "engine.cuh"
#include "graph_replay.h"
#include "k2_body.cuh"
#include "sweep_common.cuh"
#include "sweep_jit.h"
#include "sweep_tiled.cuh"
#include "tdq_internal.h"

namespace tdq {

// CTA-size limit of the generic whole-state kernel (its launch bound); every
// launch of it clamps its thread count to this.
constexpr int kK2GenericThreads = 256;

template <int MF, int MB, bool GRAD>
__global__ void __launch_bounds__(kK2GenericThreads) k2_sweep_smem(SweepArgs a, const RegPass* passes, int npf, int npb,
                                                     const DOp* gdops, int ndops, const int* rec_ptr,
                                                     const int* rec_ops, int nrec) {
  k2_body<MF, MB, GRAD, InterpProg>(a, InterpProg{passes, npf, npb, nullptr}, gdops, ndops, rec_ptr, rec_ops,
                                    nrec, blockIdx.x);
}

// Register passes of M = min(mreg, k) tile bits over ops [b, e).  Gates on
// disjoint qubits commute, so a pass may take a gate ahead of earlier ones it
// shares no qubit with.  Scanning in program order, a gate joins the pass if
// none of its qubits is blocked and its non-diagonal target's tile bit is
// held or a free slot remains; a gate left out blocks its qubits for the rest
// of the scan (every later gate on them must follow it).  The next pass scans
// the gates left out, in order.  Each pass lists its gates in a valid order.
// max_slots > 0 caps the gradient slots of a pass (a gate whose angles would
// exceed it waits for the next pass, like a gate whose bit does not fit): a
// reverse pass keeps one accumulator per slot in registers beside its
// amplitudes, and large sets of them spilled registers.
static void reg_pass_schedule(const std::vector<SweepOp>& ops, int b, int e, const int8_t* loc, int k,
                              int mreg, std::vector<std::pair<std::vector<int>, std::vector<int>>>& out,
                              int max_slots = 0) {
  const int M = std::min(mreg, k);
  std::vector<int> todo;
  for (int o = b; o < e; o++) todo.push_back(o);
  while (!todo.empty()) {
    std::vector<int> bits, taken, left;
    uint64_t blocked = 0;  // global bit positions
    int nslots = 0;
    for (int o : todo) {
      const SweepOp& op = ops[o];
      const uint64_t qm = (1ull << op.p0) | (op.p1 >= 0 ? 1ull << op.p1 : 0ull);
      int ns = 0;
      for (int j = 0; j < op.nang && j < 3; j++) ns += op.slot[j] >= 0 ? 1 : 0;
      int need = -1;
      switch (op.kind) {
        case K_RZ: case K_Z: case K_CZ: case K_RZZ: break;
        case K_CNOT: need = loc[op.p1]; break;
        default: need = loc[op.p0]; break;
      }
      bool ok = (blocked & qm) == 0;
      // a pass always takes its first gate, whatever its slots
      if (ok && max_slots > 0 && !taken.empty() && nslots + ns > max_slots) ok = false;
      if (ok && need >= 0 && std::find(bits.begin(), bits.end(), need) == bits.end()) {
        if ((int)bits.size() < M) bits.push_back(need);
        else ok = false;
      }
      if (ok) {
        nslots += ns;
        taken.push_back(o);
      } else {
        blocked |= qm;
        left.push_back(o);
      }
    }
    for (int l = 0; l < k && (int)bits.size() < M; l++)
      if (std::find(bits.begin(), bits.end(), l) == bits.end()) bits.push_back(l);
    std::sort(bits.begin(), bits.end());
    out.push_back({taken, bits});
    todo.swap(left);
  }
}

void build_program(const std::vector<SweepOp>& ops, int b, int e, const int8_t* loc, int k, bool fuse,
                   int rec0, int mreg, Program& P) {
  std::vector<std::pair<std::vector<int>, std::vector<int>>> ranges;
  reg_pass_schedule(ops, b, e, loc, k, mreg, ranges, fuse ? 0 : kRevPassSlots);
  const int M = std::min(mreg, k);
  for (const auto& rg : ranges) {
    const std::vector<int>& lb = rg.second;
    RegPass rp{};
    rp.m = (int8_t)M;
    for (int i = 0; i < kMaxRegBits; i++) rp.lb[i] = (int8_t)(i < M ? lb[i] : 0);
    rp.op_begin = (int)P.dops.size();
    auto decode = [&](int pos, int8_t* r, int8_t* l, int8_t* pp) {
      *r = -1;
      *l = -1;
      *pp = (int8_t)pos;
      if (pos < 0) return;
      const int lo = loc[pos];
      for (int i = 0; i < M; i++)
        if (lb[i] == lo) *r = (int8_t)i;
      if (*r < 0) *l = (int8_t)lo;
    };
    // one-qubit blocks open per position: index of their DOp and member list
    std::vector<int> open_dop(64, -1);
    std::vector<std::vector<int>> members;
    std::vector<int> member_dop;
    for (int o : rg.first) {
      const SweepOp& op = ops[o];
      const bool one = op.p1 < 0;
      if (fuse && one && open_dop[op.p0] >= 0) {
        members[open_dop[op.p0]].push_back(o);
        continue;
      }
      DOp d{};
      d.kind = (uint8_t)op.kind;
      decode(op.p0, &d.r0, &d.l0, &d.p0);
      decode(op.p1, &d.r1, &d.l1, &d.p1);
      d.nang = fuse ? 0 : (uint8_t)op.nang;
      for (int j = 0; j < 3; j++) d.slot[j] = (int16_t)(fuse ? -1 : op.slot[j]);
      P.dops.push_back(d);
      members.push_back({o});
      member_dop.push_back((int)P.dops.size() - 1);
      if (fuse && one) open_dop[op.p0] = (int)members.size() - 1;
      if (!one) {  // a two-qubit gate closes the blocks on its qubits
        open_dop[op.p0] = -1;
        open_dop[op.p1] = -1;
      }
    }
    for (size_t i = 0; i < members.size(); i++) {
      DOp& d = P.dops[member_dop[i]];
      if (members[i].size() > 1) {
        bool diag = true;
        for (int o : members[i]) diag = diag && (ops[o].kind == K_RZ || ops[o].kind == K_Z);
        d.kind = (uint8_t)(diag ? K_RZ : K_FUSED);
      }
      d.mat = (int16_t)((int)P.rec_ptr.size() - 1 - rec0);
      for (int o : members[i]) P.rec_ops.push_back(o);
      P.rec_ptr.push_back((int)P.rec_ops.size());
    }
    rp.op_end = (int)P.dops.size();
    P.passes.push_back(rp);
  }
}

// grads[b][s] = sum over shifted angles j of slot s of 1/2 (F(+) - F(-))
__global__ void k_param_shift_combine(const double* F, int copies, const int* slot_ptr,
                                      const int* slot_ang, int P, int B, float* grads) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * P) return;
  const int64_t b = i / P;
  const int s = (int)(i % P);
  double acc = 0.0;
  for (int e = slot_ptr[s]; e < slot_ptr[s + 1]; e++) {
    const int j = slot_ang[e];
    acc += 0.5 * (F[b * copies + 2 * j + 1] - F[b * copies + 2 * j + 2]);
  }
  grads[i] = (float)acc;
}

// ------------------------------------------------------------------ host side

struct SweepExec final : tdq_exec {
  int dev = 0, n = 0, B = 0, P = 0, F = 0, G = 0, T = 0, ng = 0, A = 0;
  int output = 0, grad = 0, NA = 0, copies = 1;
  bool smem_path = true;
  size_t smem_bytes = 0;
  int last_launches = 0;
  cudaStream_t last_stream = nullptr;
  double flops_row = 0, bytes_row = 0;
  int kclass = 0;

  SweepOp* d_ops = nullptr;
  TermDev* d_terms = nullptr;
  int* d_group_ptr = nullptr;
  uint32_t* d_amp = nullptr;
  int* d_status = nullptr;
  int* d_ps_gate = nullptr;
  int* d_ps_ang = nullptr;
  int* d_slot_ptr = nullptr;
  int* d_slot_ang = nullptr;
  double* d_ps_F = nullptr;
  RegPass* d_passes = nullptr;
  float* d_odiag = nullptr;  // observable diagonal per group [ng][2^n] (whole state; tiled when small)
  DOp* d_dops = nullptr;
  int* d_rec_ptr = nullptr;
  int* d_rec_ops = nullptr;
  int npf = 0, npb = 0, ndops = 0, nrec = 0, M = 3, threads = 32;
  int cfg_fb = 0, cfg_rb = 0;  // register bits the program was built with
  const void* spec_kernel = nullptr;  // specialised K2 program, or NULL (interpreted)
  const c2* init = nullptr;           // caller's initial states, or NULL (|0...0>)
  int64_t init_stride = 0;
  TiledSweep tiled;

  ~SweepExec() override {
    cudaFree(d_ops);
    cudaFree(d_terms);
    cudaFree(d_group_ptr);
    cudaFree(d_amp);
    cudaFree(d_status);
    cudaFree(d_ps_gate);
    cudaFree(d_ps_ang);
    cudaFree(d_slot_ptr);
    cudaFree(d_slot_ang);
    cudaFree(d_ps_F);
    cudaFree(d_passes);
    cudaFree(d_odiag);
    cudaFree(d_dops);
    cudaFree(d_rec_ptr);
    cudaFree(d_rec_ops);
    tiled_free(tiled);
  }

  tdq_status execute(const float* params, int64_t pstride, const float* inputs, double* values,
                     const double* gw, float* grads, void* stream) override {
    if (!values) return fail(TDQ_ERR_ARG, "tdq_execute: values is NULL");
    if (P > 0 && !params) return fail(TDQ_ERR_ARG, "tdq_execute: params is NULL");
    if (F > 0 && !inputs) return fail(TDQ_ERR_ARG, "tdq_execute: inputs is NULL");
    if (pstride != 0 && pstride < P) return fail(TDQ_ERR_ARG, "tdq_execute: params_stride < P");
    if (grad != TDQ_GRAD_NONE && !grads) return fail(TDQ_ERR_ARG, "tdq_execute: grads is NULL");
    if (grad == TDQ_GRAD_NONE && grads)
      return fail(TDQ_ERR_ARG, "tdq_execute: grads given to an exec compiled without gradients");
    TDQ_CUDA_TRY(cudaSetDevice(dev));
    cudaStream_t st = (cudaStream_t)stream;
    last_stream = st;
    SweepArgs a{};
    a.ops = d_ops; a.G = G; a.n = n;
    a.params = params; a.pstride = pstride; a.inputs = inputs; a.F = F;
    a.terms = d_terms; a.group_ptr = d_group_ptr; a.T = T; a.n_groups = ng;
    a.amp_idx = d_amp; a.A = A; a.output = output;
    a.values = values; a.gw = gw; a.grads = grads; a.P = P; a.status = d_status;
    a.ps_copies = copies; a.ps_gate = d_ps_gate; a.ps_ang = d_ps_ang; a.ps_F = d_ps_F;
    a.odiag = d_odiag;
    a.init = init;
    a.init_stride = init_stride;
    last_launches = 0;
    if (smem_path) {
      const unsigned grid = (unsigned)((int64_t)B * copies);
      const bool adj = grad == TDQ_GRAD_ADJOINT;
      if (spec_kernel) {
        int nd0 = 0;
        void* args[] = {&a, &d_dops, &nd0, &d_rec_ptr, &d_rec_ops, &nrec};
        TDQ_CUDA_TRY(cudaLaunchKernel(spec_kernel, dim3(grid), dim3(threads), args, smem_bytes, st));
      } else {
#define TDQ_K2(MF, MB, GG) k2_sweep_smem<MF, MB, GG><<<grid, threads, smem_bytes, st>>>(a, d_passes, npf, npb, d_dops, ndops, d_rec_ptr, d_rec_ops, nrec)
      if (M >= 4) { if (adj) TDQ_K2(4, 3, true); else TDQ_K2(4, 3, false); }
      else if (M == 3) { if (adj) TDQ_K2(3, 3, true); else TDQ_K2(3, 3, false); }
      else if (M == 2) { if (adj) TDQ_K2(2, 2, true); else TDQ_K2(2, 2, false); }
      else { if (adj) TDQ_K2(1, 1, true); else TDQ_K2(1, 1, false); }
#undef TDQ_K2
      }
      last_launches++;
      TDQ_CUDA_TRY(cudaGetLastError());
      if (grad == TDQ_GRAD_PARAM_SHIFT) {
        const int64_t tot = (int64_t)B * P;
        if (tot > 0) {
          k_param_shift_combine<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
              d_ps_F, copies, d_slot_ptr, d_slot_ang, P, B, grads);
          last_launches++;
        }
        TDQ_CUDA_TRY(cudaGetLastError());
      }
      return ok();
    }
    tdq_status s = tiled_execute(tiled, a, grad, st, &last_launches);
    if (s != TDQ_OK) return s;
    if (grad == TDQ_GRAD_PARAM_SHIFT) {
      const int64_t tot = (int64_t)B * P;
      if (tot > 0) {
        k_param_shift_combine<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
            d_ps_F, copies, d_slot_ptr, d_slot_ang, P, B, grads);
        last_launches++;
      }
      TDQ_CUDA_TRY(cudaGetLastError());
    }
    return ok();
  }

  tdq_status set_initial_state(const float* psi0, int64_t stride) override {
    if (stride != 0 && stride < ((int64_t)1 << n))
      return fail(TDQ_ERR_ARG, "tdq_exec_set_initial_state: row_stride must be 0 or >= 2^n");
    if (stride < 0) return fail(TDQ_ERR_ARG, "tdq_exec_set_initial_state: negative row_stride");
    init = reinterpret_cast<const c2*>(psi0);
    init_stride = psi0 ? stride : 0;
    return ok();
  }

  tdq_status status() override {
    TDQ_CUDA_TRY(cudaSetDevice(dev));
    TDQ_CUDA_TRY(cudaStreamSynchronize(last_stream));
    int h = 0;
    TDQ_CUDA_TRY(cudaMemcpy(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost));
    TDQ_CUDA_TRY(cudaMemset(d_status, 0, sizeof(int)));
    if (h & (1 << TDQ_ERR_TIMEOUT)) return fail(TDQ_ERR_TIMEOUT, "a device wait timed out");
    if (h & (1 << TDQ_ERR_NONFINITE)) return fail(TDQ_ERR_NONFINITE, "non-finite parameter or input");
    return ok();
  }

  int launches() const override { return last_launches; }

  // per launch unit of the first row chunk of a tiled sweep (see TiledSweep)
  tdq_status timings(float* ms, int max, int* n) override {
    if (smem_path || tiled.ev.empty())
      return fail(TDQ_ERR_STATE, "tdq_exec_timings: a tiled sweep compiled with record_timings only");
    const int units = (int)tiled.ev.size() / 2;
    if (n) *n = units;
    if (!ms) return ok();
    if (max < units) return fail(TDQ_ERR_ARG, "tdq_exec_timings: buffer too small");
    TDQ_CUDA_TRY(cudaSetDevice(dev));
    TDQ_CUDA_TRY(cudaStreamSynchronize(last_stream));
    for (int u = 0; u < units; u++) TDQ_CUDA_TRY(cudaEventElapsedTime(&ms[u], tiled.ev[2 * u], tiled.ev[2 * u + 1]));
    return ok();
  }

  tdq_status launch_work(double* flops, double* bytes, int* kind, int max, int* n) const override {
    if (smem_path) return fail(TDQ_ERR_UNSUPPORTED, "tdq_exec_launch_work: tiled state sweeps only");
    const int units = (int)tiled.unit_kind.size();
    if (n) *n = units;
    if (!flops && !bytes && !kind) return ok();
    if (max < units) return fail(TDQ_ERR_ARG, "tdq_exec_launch_work: buffer too small");
    const double rows = (double)std::min(tiled.chunk_rows, tiled.rows);
    for (int u = 0; u < units; u++) {
      if (flops) flops[u] = tiled.unit_flops[u] * rows;
      if (bytes) bytes[u] = tiled.unit_bytes[u] * rows;
      if (kind) kind[u] = tiled.unit_kind[u];
    }
    return ok();
  }

  void work(double* f, double* by, int* k) const override {
    *f = flops_row;
    *by = bytes_row;
    *k = kclass;
  }

  tdq_status config(int* c4) const override {
    if (smem_path) {
      c4[0] = threads;
      c4[1] = spec_kernel ? cfg_fb : M;
      c4[2] = spec_kernel ? cfg_rb : kRevRegBits;
      c4[3] = 0;
    } else {
      c4[0] = tiled.nthreads;
      c4[1] = tiled.fb;
      c4[2] = tiled.rb;
      c4[3] = tiled.k;
    }
    return ok();
  }
};

template <typename T>
static tdq_status upload(T** dst, const std::vector<T>& v) {
  *dst = nullptr;
  if (v.empty()) return TDQ_OK;
  cudaError_t e = cudaMalloc((void**)dst, sizeof(T) * v.size());
  if (e != cudaSuccess) return fail(TDQ_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(TDQ_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
  return TDQ_OK;
}

// Algorithmic FP32 work of one row, by the counting rule of the design notes:
// a dense 2x2 complex gate on a pair 28 flops, a diagonal phase 6 flops per
// amplitude, permutations and sign flips 0; the observable 3 + 2T per
// amplitude; the reverse sweep twice the forward plus the gradient dots.
static double sweep_flops(const tdq_circuit* c, bool adjoint, const std::vector<int>& tail) {
  const double dim = std::ldexp(1.0, c->n);
  double fwd = 0, grad_dots = 0;
  std::vector<char> folded(c->gates.size(), 0);
  for (int gi : tail) folded[gi] = 1;  // closed with the observable: no work on the state
  for (size_t gi = 0; gi < c->gates.size(); gi++) {
    if (folded[gi]) continue;
    fwd += gate_fwd_flops(c->gates[gi].kind, dim);
    grad_dots += gate_dot_flops(c->gates[gi].kind, dim);
  }
  const double obs = (3.0 + 2.0 * (double)c->terms.size()) * dim;
  return adjoint ? 3 * fwd + grad_dots + 2 * obs : fwd + obs;
}

// Gates at the end of the circuit that the expectation network can close
// with the observable first: parameter-free CNOT, CZ, X, Y and Z map every
// Z-product term to a Z-product term (G^dagger Z..Z G), so contracting G and
// its conjugate into the observable tensors before the rest of the network
// is an exact change of contraction order (Sec. 3.2.1: the order changes only
// the cost).  A gate qualifies when every later gate that stays acts on other
// qubits (it commutes to the end).  Returns the qualifying gates, last first
// (the order in which they are folded into the terms); the first gate of the
// circuit always stays.
static std::vector<int> clifford_tail(const tdq_circuit* c) {
  std::vector<int> tail;
  uint64_t blocked = 0;
  for (int gi = (int)c->gates.size() - 1; gi >= 1; gi--) {
    const GateRec& g = c->gates[gi];
    const uint64_t qm = (1ull << g.q[0]) | (g.q[1] >= 0 ? 1ull << g.q[1] : 0ull);
    const bool kind_ok = g.kind == TDQ_CNOT || g.kind == TDQ_CZ || g.kind == TDQ_X || g.kind == TDQ_Y ||
                         g.kind == TDQ_Z;
    if (kind_ok && !(blocked & qm)) tail.push_back(gi);
    else blocked |= qm;
  }
  return tail;
}

// Fold the tail gates (last first) into Z-product terms on bit positions
// (position n-1-q of qubit q): CNOT(c -> t) maps Z_t to Z_c Z_t, X and Y
// negate Z on their qubit, CZ and Z commute with every term.
static void fold_tail_into_terms(const tdq_circuit* c, const std::vector<int>& tail, std::vector<TermDev>& terms) {
  for (int gi : tail) {
    const GateRec& g = c->gates[gi];
    const uint32_t b0 = 1u << (c->n - 1 - g.q[0]);
    for (TermDev& t : terms) {
      if (g.kind == TDQ_CNOT && (t.pmask_lo & (1u << (c->n - 1 - g.q[1])))) t.pmask_lo ^= b0;
      if ((g.kind == TDQ_X || g.kind == TDQ_Y) && (t.pmask_lo & b0)) t.coeff = -t.coeff;
    }
  }
}

// The circuit's gates as device ops (bit positions, angle sources, gradient
// slots); ps_gate / ps_ang list the (op, angle) pairs with a parameter.
// Gates listed in `skip` (the Clifford tail of an expectation program) are
// left out.
static std::vector<SweepOp> sweep_ops(const tdq_circuit* c, std::vector<int>* ps_gate, std::vector<int>* ps_ang,
                                      const std::vector<int>* skip = nullptr) {
  std::vector<SweepOp> ops;
  std::vector<char> drop(c->gates.size(), 0);
  if (skip)
    for (int gi : *skip) drop[gi] = 1;
  for (int gi = 0; gi < (int)c->gates.size(); gi++) {
    if (drop[gi]) continue;
    const GateRec& g = c->gates[gi];
    SweepOp op{};
    op.kind = (int8_t)g.kind;
    op.p0 = (int8_t)(c->n - 1 - g.q[0]);
    op.p1 = (int8_t)(g.q[1] >= 0 ? c->n - 1 - g.q[1] : -1);
    op.nang = (int8_t)gate_n_angles(g.kind);
    for (int j = 0; j < 3; j++) {
      op.src[j] = g.src[j];
      op.fixed[j] = (float)g.fixed[j];
      op.slot[j] = (j < op.nang && g.src[j] >= 0) ? g.src[j] : -1;
      if (j < op.nang && g.src[j] >= 0) {
        ps_gate->push_back((int)ops.size());
        ps_ang->push_back(j);
      }
    }
    ops.push_back(op);
  }
  return ops;
}

// Bytes of one row's outputs (FP64 values).
static double out_bytes_row(int output, int n, int A, int ng) {
  switch (output) {
    case TDQ_OUT_AMPLITUDE: return 16.0 * A;
    case TDQ_OUT_STATE: return std::ldexp(16.0, n);
    case TDQ_OUT_PROBS: return std::ldexp(8.0, n);
    default: return 8.0 * ng;
  }
}

// Threads per CTA of the whole-state kernel for n qubits and M forward bits:
// one thread per register group up to 256 (the autotuner's pick for the
// 12-qubit classifier with the packed register kernels: 2.00 M against
// 1.92 M evals/s at 512 threads; 512 had won before the packing shortened
// the program).
static int k2_threads(int n, int M) { return std::max(32, std::min(256, (1 << n) >> M)); }

// Source of the specialised whole-state kernel of circuit c (adjoint: with
// the reverse program).
static void k2_program(const tdq_circuit* c, bool adj, int fb, int rb, Program& prog, int* npf, int* npb,
                       bool peel) {
  std::vector<int> psg, psa;
  const std::vector<int> tail = peel ? clifford_tail(c) : std::vector<int>();
  const std::vector<SweepOp> ops = sweep_ops(c, &psg, &psa, &tail);
  int8_t loc[32];
  for (int p = 0; p < 32; p++) loc[p] = (int8_t)(p < c->n ? p : -1);
  build_program(ops, 0, (int)ops.size(), loc, c->n, true, 0, fb, prog);
  *npf = (int)prog.passes.size();
  if (adj) build_program(ops, 0, (int)ops.size(), loc, c->n, false, 0, rb, prog);
  *npb = (int)prog.passes.size() - *npf;
}

static std::string k2_source(const tdq_circuit* c, bool adj, int fb, int rb, Program& prog, int* npf, int* npb,
                             bool peel) {
  k2_program(c, adj, fb, rb, prog, npf, npb, peel);
  const int M = std::min(fb, c->n);
  return k2_specialised_source(prog, *npf, *npb, M, std::min(rb, c->n), k2_threads(c->n, M),
                               c->n_params, c->n, "tdq_k2_specialised");
}

// Part of a multi-circuit launch: the circuit's tables only (its program is
// compiled with the other circuits'), for a CTA of `threads` threads.
struct MultiHook {
  int threads;
};

static tdq_status compile_sweep_impl(const tdq_circuit* c, const tdq_compile_opts* o, tdq_exec** out,
                                     MultiHook* hook, int threads_override = 0);
static tdq_status sweep_autotune(const tdq_circuit* c, const tdq_compile_opts* o, tdq_exec** out);

}  // namespace tdq

extern "C" tdq_status tdq_compile_sweep(const tdq_circuit* c, const tdq_compile_opts* o, tdq_exec** out) {
  if (o && o->autotune) return tdq::sweep_autotune(c, o, out);
  return tdq::compile_sweep_impl(c, o, out, nullptr);
}

namespace tdq {

static tdq_status compile_sweep_impl(const tdq_circuit* c, const tdq_compile_opts* o, tdq_exec** out,
                                     MultiHook* hook, int threads_override) {
  if (!c || !o || !out) return fail(TDQ_ERR_ARG, "tdq_compile_sweep: NULL argument");
  *out = nullptr;
  if (o->batch < 1) return fail(TDQ_ERR_ARG, "tdq_compile_sweep: batch must be >= 1");
  if (o->output < TDQ_OUT_EXPVAL || o->output > TDQ_OUT_PROBS)
    return fail(TDQ_ERR_ARG, "tdq_compile_sweep: bad output kind");
  if (o->grad < TDQ_GRAD_NONE || o->grad > TDQ_GRAD_PARAM_SHIFT)
    return fail(TDQ_ERR_ARG, "tdq_compile_sweep: bad gradient mode");
  if (o->grad != TDQ_GRAD_NONE && o->output != TDQ_OUT_EXPVAL)
    return fail(TDQ_ERR_UNSUPPORTED, "tdq_compile_sweep: gradients need expectation outputs");
  if (c->n > 30) return fail(TDQ_ERR_UNSUPPORTED, "tdq_compile_sweep: more than 30 qubits");
  if (o->output == TDQ_OUT_EXPVAL && c->n_groups == 0)
    return fail(TDQ_ERR_STATE, "tdq_compile_sweep: circuit has no observable");
  if (o->output == TDQ_OUT_AMPLITUDE && c->amps.empty())
    return fail(TDQ_ERR_STATE, "tdq_compile_sweep: circuit has no amplitude request");

  SweepExec* e = new (std::nothrow) SweepExec();
  if (!e) return fail(TDQ_ERR_OOM, "tdq_compile_sweep: host allocation");
  auto bail = [&](tdq_status s) {
    delete e;
    return s;
  };
  e->dev = o->device;
  if (cudaSetDevice(e->dev) != cudaSuccess) return bail(fail(TDQ_ERR_CUDA, "cudaSetDevice failed"));
  e->n = c->n;
  e->B = o->batch;
  e->P = c->n_params;
  e->F = c->n_inputs;
  e->G = (int)c->gates.size();
  e->ng = c->n_groups;
  e->A = (int)c->amps.size();
  e->output = o->output;
  e->grad = o->grad;

  std::vector<int> ps_gate, ps_ang;
  // expectation programs: the Clifford tail is folded into the terms
  const std::vector<int> tail = o->output == TDQ_OUT_EXPVAL ? clifford_tail(c) : std::vector<int>();
  const std::vector<SweepOp> ops = sweep_ops(c, &ps_gate, &ps_ang, &tail);
  e->G = (int)ops.size();
  // terms sorted by group
  std::vector<TermDev> terms;
  std::vector<int> gptr(e->ng + 1, 0);
  for (int g = 0; g < e->ng; g++) {
    gptr[g] = (int)terms.size();
    for (const Term& t : c->terms) {
      if (t.group != g) continue;
      TermDev d{};
      for (int q : t.zq) {
        const int p = c->n - 1 - q;
        if (p < 32) d.pmask_lo |= 1u << p;
        else d.pmask_hi |= 1u << (p - 32);
      }
      d.coeff = (float)t.coeff;
      d.group = g;
      terms.push_back(d);
    }
  }
  gptr[e->ng] = (int)terms.size();
  fold_tail_into_terms(c, tail, terms);
  e->T = (int)terms.size();
  std::vector<uint32_t> amp;
  for (const auto& bits : c->amps) {
    uint32_t x = 0;
    for (int q = 0; q < c->n; q++) x = (x << 1) | bits[q];
    amp.push_back(x);
  }
  tdq_status s;
  if ((s = upload(&e->d_ops, ops)) != TDQ_OK) return bail(s);
  if ((s = upload(&e->d_terms, terms)) != TDQ_OK) return bail(s);
  if ((s = upload(&e->d_group_ptr, gptr)) != TDQ_OK) return bail(s);
  if ((s = upload(&e->d_amp, amp)) != TDQ_OK) return bail(s);
  if (cudaMalloc(&e->d_status, sizeof(int)) != cudaSuccess) return bail(fail(TDQ_ERR_OOM, "status word"));
  cudaMemset(e->d_status, 0, sizeof(int));

  if (o->grad == TDQ_GRAD_PARAM_SHIFT) {
    e->NA = (int)ps_gate.size();
    e->copies = 1 + 2 * e->NA;
    std::vector<int> sptr(e->P + 1, 0), sang;
    for (int sl = 0; sl < e->P; sl++) {
      sptr[sl] = (int)sang.size();
      for (int j = 0; j < e->NA; j++)
        if (ops[ps_gate[j]].slot[ps_ang[j]] == sl) sang.push_back(j);
    }
    sptr[e->P] = (int)sang.size();
    if ((s = upload(&e->d_ps_gate, ps_gate)) != TDQ_OK) return bail(s);
    if ((s = upload(&e->d_ps_ang, ps_ang)) != TDQ_OK) return bail(s);
    if ((s = upload(&e->d_slot_ptr, sptr)) != TDQ_OK) return bail(s);
    if ((s = upload(&e->d_slot_ang, sang)) != TDQ_OK) return bail(s);
    if (cudaMalloc(&e->d_ps_F, sizeof(double) * (size_t)e->B * e->copies) != cudaSuccess)
      return bail(fail(TDQ_ERR_OOM, "parameter-shift buffer"));
  }

  const bool adj = o->grad == TDQ_GRAD_ADJOINT;
  if (o->fwd_reg_bits < 0 || o->fwd_reg_bits > 4 || o->rev_reg_bits < 0 || o->rev_reg_bits > 4)
    return bail(fail(TDQ_ERR_ARG, "tdq_compile_sweep: register bits must be in 1..4 (0 = default)"));
  if (o->interpret && (o->fwd_reg_bits || o->rev_reg_bits))
    return bail(fail(TDQ_ERR_ARG, "tdq_compile_sweep: register bits apply to specialised programs only"));
  // register bits: specialised whole-state programs default to narrow passes
  // (short per-gate code, re-run by more groups: the instruction footprint
  // decides their speed); tiled and generic programs to 4 / 3
  const bool k2spec = !o->interpret;
  const int fb = o->fwd_reg_bits ? o->fwd_reg_bits : (k2spec ? kSpecFwdRegBits : kFwdRegBits);
  const int rb = o->rev_reg_bits ? o->rev_reg_bits : (k2spec ? kSpecRevRegBits : kRevRegBits);
  // tiled programs: the generic kernels are compiled for kFwdRegBits /
  // kRevRegBits; specialised ones take their own defaults
  const int fb1 = o->fwd_reg_bits ? o->fwd_reg_bits : (o->interpret ? kFwdRegBits : kTiledSpecFwdRegBits);
  const int rb1 = o->rev_reg_bits ? o->rev_reg_bits : (o->interpret ? kRevRegBits : kTiledSpecRevRegBits);
  e->cfg_fb = fb;
  e->cfg_rb = rb;
  const int smem_max_n = o->max_smem_qubits > 0 ? o->max_smem_qubits : (adj ? 13 : 14);
  e->smem_path = c->n <= smem_max_n;
  e->flops_row = sweep_flops(c, adj, tail);
  if (o->grad == TDQ_GRAD_PARAM_SHIFT) e->flops_row *= e->copies;
  Program prog;
  if (e->smem_path) {
    int8_t loc[32];
    for (int p = 0; p < 32; p++) loc[p] = (int8_t)(p < c->n ? p : -1);
    build_program(ops, 0, (int)ops.size(), loc, c->n, true, 0, fb, prog);
    e->npf = (int)prog.passes.size();
    if (adj) build_program(ops, 0, (int)ops.size(), loc, c->n, false, 0, rb, prog);
    e->npb = (int)prog.passes.size() - e->npf;
    e->ndops = (int)prog.dops.size();
    e->nrec = (int)prog.rec_ptr.size() - 1;
    const size_t dim = (size_t)1 << c->n;
    e->smem_bytes = dim * sizeof(c2) * (adj ? 2 : 1) + sizeof(OpMat) * e->nrec + sizeof(DOp) * e->ndops +
                    (adj ? sizeof(double) * e->P : 0) + 32 * sizeof(double) + 16;
    if (e->smem_bytes > 227 * 1024) e->smem_path = false;
  }
  if (hook && !e->smem_path)
    return bail(fail(TDQ_ERR_UNSUPPORTED, "tdq_compile_multi: a circuit's state does not fit one CTA's shared memory"));
  if (e->smem_path) {
    e->M = std::min(fb, c->n);
    e->threads = hook ? hook->threads : (threads_override > 0 ? threads_override : k2_threads(c->n, e->M));
    if ((s = upload(&e->d_passes, prog.passes)) != TDQ_OK) return bail(s);
    if (e->output == TDQ_OUT_EXPVAL) {  // D_g[x] = sum_{t in g} c_t (-1)^{popc(x & mask_t)}
      const size_t dim = (size_t)1 << c->n;
      std::vector<float> od((size_t)e->ng * dim);
      for (int g = 0; g < e->ng; g++)
        for (size_t x = 0; x < dim; x++) {
          double d = 0.0;
          for (int t = gptr[g]; t < gptr[g + 1]; t++)
            d += (__builtin_popcount((unsigned)x & terms[t].pmask_lo) & 1) ? -(double)terms[t].coeff : (double)terms[t].coeff;
          od[(size_t)g * dim + x] = (float)d;
        }
      if ((s = upload(&e->d_odiag, od)) != TDQ_OK) return bail(s);
    }
    if ((s = upload(&e->d_dops, prog.dops)) != TDQ_OK) return bail(s);
    if ((s = upload(&e->d_rec_ptr, prog.rec_ptr)) != TDQ_OK) return bail(s);
    if ((s = upload(&e->d_rec_ops, prog.rec_ops)) != TDQ_OK) return bail(s);
    cudaError_t ce = cudaSuccess;
    if (!o->interpret) {
      // specialised program: no decoded ops in shared memory; per-warp FP32
      // gradient rows instead of FP64 sums
      const size_t dim = (size_t)1 << c->n;
      const size_t gb = adj ? k2_grad_bytes(true, e->P, e->threads) : 0;
      const size_t sb = dim * sizeof(c2) * (adj ? 2 : 1) + sizeof(OpMat) * e->nrec + ((gb + 7) & ~(size_t)7) +
                        32 * sizeof(double) + 16;
      if (hook) {  // compiled later with the other circuits of the launch
        if (sb > 227 * 1024)
          return bail(fail(TDQ_ERR_UNSUPPORTED, "tdq_compile_multi: a circuit's program does not fit shared memory"));
        e->smem_bytes = sb;
        e->kclass = 2;
        e->bytes_row = 4.0 * e->P + 4.0 * e->F + out_bytes_row(e->output, c->n, e->A, e->ng) + (adj ? 4.0 * e->P : 0);
        *out = e;
        return ok();
      }
      if (sb <= 227 * 1024) {
        const std::string src = k2_specialised_source(prog, e->npf, e->npb, e->M, std::min(rb, c->n),
                                                      e->threads, e->P, c->n, "tdq_k2_specialised");
        if ((s = jit_kernel(src, "tdq_k2_specialised", &e->spec_kernel)) != TDQ_OK) return bail(s);
        e->smem_bytes = sb;
        ce = cudaFuncSetAttribute(e->spec_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
        if (ce != cudaSuccess)
          return bail(fail(TDQ_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce)));
      }
    }
    if (!e->spec_kernel && (fb != kFwdRegBits || rb != kRevRegBits)) {
      // the specialised program did not fit: the generic kernels' program
      if (o->fwd_reg_bits || o->rev_reg_bits)
        return bail(fail(TDQ_ERR_UNSUPPORTED, "tdq_compile_sweep: register bits need a specialised program"));
      prog = Program{};
      int8_t loc[32];
      for (int p = 0; p < 32; p++) loc[p] = (int8_t)(p < c->n ? p : -1);
      build_program(ops, 0, (int)ops.size(), loc, c->n, true, 0, kFwdRegBits, prog);
      e->npf = (int)prog.passes.size();
      if (adj) build_program(ops, 0, (int)ops.size(), loc, c->n, false, 0, kRevRegBits, prog);
      e->npb = (int)prog.passes.size() - e->npf;
      e->ndops = (int)prog.dops.size();
      e->nrec = (int)prog.rec_ptr.size() - 1;
      e->M = std::min(kFwdRegBits, c->n);
      e->threads = k2_threads(c->n, e->M);
      const size_t dim = (size_t)1 << c->n;
      e->smem_bytes = dim * sizeof(c2) * (adj ? 2 : 1) + sizeof(OpMat) * e->nrec + sizeof(DOp) * e->ndops +
                      (adj ? sizeof(double) * e->P : 0) + 32 * sizeof(double) + 16;
      cudaFree(e->d_passes);
      cudaFree(e->d_dops);
      cudaFree(e->d_rec_ptr);
      cudaFree(e->d_rec_ops);
      e->d_passes = nullptr;
      e->d_dops = nullptr;
      e->d_rec_ptr = e->d_rec_ops = nullptr;
      if ((s = upload(&e->d_passes, prog.passes)) != TDQ_OK) return bail(s);
      if ((s = upload(&e->d_dops, prog.dops)) != TDQ_OK) return bail(s);
      if ((s = upload(&e->d_rec_ptr, prog.rec_ptr)) != TDQ_OK) return bail(s);
      if ((s = upload(&e->d_rec_ops, prog.rec_ops)) != TDQ_OK) return bail(s);
    }
    // the generic kernel's launch bound caps its CTA size (the specialised
    // kernel is compiled for e->threads)
    if (!e->spec_kernel) e->threads = std::min(e->threads, kK2GenericThreads);
#define TDQ_SETSM(MF, MB, GG) ce = cudaFuncSetAttribute(k2_sweep_smem<MF, MB, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e->smem_bytes)
    if (e->spec_kernel) {
    } else if (e->M >= 4) { if (adj) TDQ_SETSM(4, 3, true); else TDQ_SETSM(4, 3, false); }
    else if (e->M == 3) { if (adj) TDQ_SETSM(3, 3, true); else TDQ_SETSM(3, 3, false); }
    else if (e->M == 2) { if (adj) TDQ_SETSM(2, 2, true); else TDQ_SETSM(2, 2, false); }
    else { if (adj) TDQ_SETSM(1, 1, true); else TDQ_SETSM(1, 1, false); }
#undef TDQ_SETSM
    if (ce != cudaSuccess) return bail(fail(TDQ_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce)));
    e->kclass = 2;
    // compulsory HBM bytes per row: parameters, inputs, outputs, gradients
    e->bytes_row = 4.0 * e->P + 4.0 * e->F + out_bytes_row(e->output, c->n, e->A, e->ng) + (adj ? 4.0 * e->P : 0);
  }
  if (!e->smem_path) {
    // the observable's diagonal per output group, read by the last tile pass
    // instead of evaluating every term per amplitude: kept while the tables
    // stay small enough to live in L2 (at most 64 MiB)
    if (e->output == TDQ_OUT_EXPVAL && (std::ldexp((double)e->ng * 4.0, c->n) <= 64.0 * 1024 * 1024)) {
      const size_t dim = (size_t)1 << c->n;
      std::vector<float> od((size_t)e->ng * dim);
      for (int g = 0; g < e->ng; g++)
        for (size_t x = 0; x < dim; x++) {
          double d = 0.0;
          for (int t = gptr[g]; t < gptr[g + 1]; t++)
            d += (__builtin_popcount((unsigned)x & terms[t].pmask_lo) & 1) ? -(double)terms[t].coeff
                                                                          : (double)terms[t].coeff;
          od[(size_t)g * dim + x] = (float)d;
        }
      if ((s = upload(&e->d_odiag, od)) != TDQ_OK) return bail(s);
    }
    s = tiled_compile(e->tiled, c, ops, ps_gate, e->B * e->copies, adj, o->tile_qubits, o->interpret != 0, fb1, rb1,
                      &e->bytes_row);
    if (s != TDQ_OK) return bail(s);
    // outputs: the state read back from HBM and written out as values
    if (e->output == TDQ_OUT_STATE || e->output == TDQ_OUT_PROBS)
      e->bytes_row += std::ldexp(8.0, c->n) + out_bytes_row(e->output, c->n, e->A, e->ng);
    e->kclass = 1;
    if (o->record_timings) {  // events around every launch unit of the first row chunk
      e->tiled.ev.assign(2 * e->tiled.unit_kind.size(), nullptr);
      for (cudaEvent_t& ev : e->tiled.ev)
        if (cudaEventCreate(&ev) != cudaSuccess) return bail(fail(TDQ_ERR_CUDA, "tiled sweep: timing events"));
    }
  }
  *out = e;
  return ok();
}

// A buffer twice the L2 size, written before every timed run so that each run
// starts cold (kernel code and tables from HBM), as the benchmark measures.
struct L2Flush {
  void* buf = nullptr;
  size_t bytes = 0;
  tdq_status init(int dev) {
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
      return fail(TDQ_ERR_CUDA, "autotune: L2 size");
    bytes = 2 * (size_t)std::max(l2, 1 << 20);
    if (cudaMalloc(&buf, bytes) != cudaSuccess) return fail(TDQ_ERR_OOM, "autotune: flush buffer");
    return TDQ_OK;
  }
  cudaError_t run(int it, cudaStream_t st) const { return cudaMemsetAsync(buf, it & 0xff, bytes, st); }
  ~L2Flush() { cudaFree(buf); }
};

// Median time (ms) of a few executions of a sweep exec on synthetic
// parameters (the kernels' work does not depend on the values), each after an
// L2 flush.
static tdq_status sweep_time(tdq_exec* ex, const tdq_circuit* c, const tdq_compile_opts* o, float* ms) {
  SweepExec* e = static_cast<SweepExec*>(ex);
  const size_t np = (size_t)std::max(1, e->B * e->P), nx = (size_t)std::max(1, e->B * e->F);
  const size_t nv = (size_t)std::max(1.0, e->B * out_bytes_row(e->output, c->n, e->A, e->ng) / 8.0);
  float *p = nullptr, *x = nullptr, *g = nullptr;
  double* v = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  auto done = [&](tdq_status s) {
    cudaFree(p);
    cudaFree(x);
    cudaFree(g);
    cudaFree(v);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    return s;
  };
  if (cudaMalloc(&p, sizeof(float) * np) != cudaSuccess || cudaMalloc(&x, sizeof(float) * nx) != cudaSuccess ||
      cudaMalloc(&g, sizeof(float) * np) != cudaSuccess || cudaMalloc(&v, sizeof(double) * nv) != cudaSuccess)
    return done(fail(TDQ_ERR_OOM, "autotune: buffers"));
  std::vector<float> h(std::max(np, nx), 0.37f);
  if (cudaMemcpy(p, h.data(), sizeof(float) * np, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(x, h.data(), sizeof(float) * nx, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
      cudaEventCreate(&b) != cudaSuccess)
    return done(fail(TDQ_ERR_CUDA, "autotune: setup"));
  L2Flush fl;
  tdq_status fs = fl.init(e->dev);
  if (fs != TDQ_OK) return done(fs);
  std::vector<float> t;
  for (int it = 0; it < 6; it++) {
    if (fl.run(it, st) != cudaSuccess || cudaEventRecord(a, st) != cudaSuccess)
      return done(fail(TDQ_ERR_CUDA, "autotune: event"));
    tdq_status s = e->execute(e->P > 0 ? p : nullptr, e->P, e->F > 0 ? x : nullptr, v, nullptr,
                              o->grad == TDQ_GRAD_NONE ? nullptr : g, st);
    if (s != TDQ_OK) return done(s);
    if (cudaEventRecord(b, st) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess)
      return done(fail(TDQ_ERR_CUDA, "autotune: run"));
    float m = 0.f;
    cudaEventElapsedTime(&m, a, b);
    if (it > 0) t.push_back(m);  // the first run warms up
  }
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  cudaMemset(e->d_status, 0, sizeof(int));
  return done(TDQ_OK);
}

// Launch configurations timed on this circuit and batch, the fastest kept:
// whole-state kernels -- CTA size 128 / 256 / 512 x register bits 2 / 3 of
// the specialised program (compiled concurrently on the host's cores); tiled
// sweeps -- tile bits 10..13.
static tdq_status sweep_autotune(const tdq_circuit* c, const tdq_compile_opts* o, tdq_exec** out) {
  if (!c || !o || !out) return fail(TDQ_ERR_ARG, "tdq_compile_sweep: NULL argument");
  *out = nullptr;
  if (o->interpret || o->fwd_reg_bits || o->rev_reg_bits || o->tile_qubits)
    return fail(TDQ_ERR_ARG, "tdq_compile_sweep: autotune picks specialised programs, register bits and tiles itself");
  const bool adj = o->grad == TDQ_GRAD_ADJOINT;
  const int smem_max_n = o->max_smem_qubits > 0 ? o->max_smem_qubits : (adj ? 13 : 14);
  struct Cand {
    int threads, bits, tile;
  };
  std::vector<Cand> cands;
  if (c->n <= smem_max_n) {
    for (int threads : {128, 256, 512})
      for (int bits : {2, 3}) cands.push_back({threads, bits, 0});
    // warm the compile cache: every candidate's kernel concurrently
    std::vector<std::thread> pool;
    for (const Cand& k : cands)
      pool.emplace_back([&, k] {
        try {
          if (cudaSetDevice(o->device) != cudaSuccess) return;
          Program prog;
          int npf = 0, npb = 0;
          k2_program(c, adj, k.bits, k.bits, prog, &npf, &npb, o->output == TDQ_OUT_EXPVAL);
          const std::string src = k2_specialised_source(prog, npf, npb, std::min(k.bits, c->n),
                                                        std::min(k.bits, c->n), k.threads, c->n_params, c->n,
                                                        "tdq_k2_specialised");
          const void* kern = nullptr;
          jit_kernel(src, "tdq_k2_specialised", &kern);  // failures surface again in the build below
        } catch (...) {  // (the build below reports it)
        }
      });
    for (auto& t : pool) t.join();
  } else {
    for (int tile = 10; tile <= std::min(13, c->n); tile++) cands.push_back({0, 0, tile});
  }
  tdq_exec* best = nullptr;
  float best_ms = 0.f;
  for (const Cand& k : cands) {
    tdq_compile_opts oc = *o;
    oc.autotune = 0;
    oc.fwd_reg_bits = k.bits;
    oc.rev_reg_bits = k.bits;
    oc.tile_qubits = k.tile;
    tdq_exec* e = nullptr;
    tdq_status s = compile_sweep_impl(c, &oc, &e, nullptr, k.threads);
    if (s == TDQ_ERR_UNSUPPORTED) continue;  // this configuration does not fit
    if (s != TDQ_OK) {
      delete best;
      return s;
    }
    float ms = 0.f;
    s = sweep_time(e, c, &oc, &ms);
    if (s != TDQ_OK) {
      delete e;
      delete best;
      return s;
    }
    if (!best || ms < best_ms) {
      delete best;
      best = e;
      best_ms = ms;
    } else {
      delete e;
    }
  }
  if (!best) return fail(TDQ_ERR_UNSUPPORTED, "tdq_compile_sweep: no launch configuration fits");
  *out = best;
  return ok();
}

}  // namespace tdq

using namespace tdq;

extern "C" tdq_status tdq_sweep_source(const tdq_circuit* c, int grad, int tile_qubits, char* buf, size_t cap,
                                       size_t* len) {
  if (!c || !len) return fail(TDQ_ERR_ARG, "tdq_sweep_source: NULL argument");
  if (grad != TDQ_GRAD_NONE && grad != TDQ_GRAD_ADJOINT)
    return fail(TDQ_ERR_ARG, "tdq_sweep_source: grad must be TDQ_GRAD_NONE or TDQ_GRAD_ADJOINT");
  const bool adj = grad == TDQ_GRAD_ADJOINT;
  std::string src;
  if (tile_qubits == 0) {
    if (c->n > 14) return fail(TDQ_ERR_UNSUPPORTED, "tdq_sweep_source: more than 14 qubits in one CTA");
    Program prog;
    int npf = 0, npb = 0;
    src = k2_source(c, adj, kSpecFwdRegBits, kSpecRevRegBits, prog, &npf, &npb, c->n_groups > 0);
  } else {
    if (c->n > 30) return fail(TDQ_ERR_UNSUPPORTED, "tdq_sweep_source: more than 30 qubits");
    std::vector<int> psg, psa;
    const std::vector<int> tail = c->n_groups > 0 ? clifford_tail(c) : std::vector<int>();
    const std::vector<SweepOp> ops = sweep_ops(c, &psg, &psa, &tail);
    TiledSweep t;
    TiledHost h;
    tdq_status s = tiled_plan(t, c, ops, psg, 1, adj, tile_qubits, kTiledSpecFwdRegBits, kTiledSpecRevRegBits, h);
    if (s != TDQ_OK) return s;
    std::vector<int> nacc;
    src = k1_specialised_source(t, h.prog, std::max(32, std::min(256, 1 << (t.k - kTiledSpecFwdRegBits))),
                                std::max(32, std::min(256, 1 << (t.k - kTiledSpecRevRegBits))), &nacc);
  }
  *len = src.size() + 1;
  if (buf) {
    if (cap < src.size() + 1) return fail(TDQ_ERR_ARG, "tdq_sweep_source: buffer too small");
    std::memcpy(buf, src.c_str(), src.size() + 1);
  }
  return ok();
}

// ------------------------------------------------- many circuits, one launch

namespace tdq {

// The shift rule over every circuit of a multi-circuit launch: entry i of the
// packed gradients belongs to the circuit whose range [begin, begin + B P)
// holds it.
struct MultiPs {
  const double* F;
  const int* slot_ptr;
  const int* slot_ang;
  int copies, P;
  int64_t begin, g_off;
};

__global__ void k_multi_ps_combine(const MultiPs* tab, int nc, int64_t total, float* grads) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  int lo = 0, hi = nc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (tab[mid].begin <= i) lo = mid;
    else hi = mid - 1;
  }
  const MultiPs t = tab[lo];
  const int64_t j = i - t.begin, b = j / t.P;
  const int s = (int)(j % t.P);
  double acc = 0.0;
  for (int e = t.slot_ptr[s]; e < t.slot_ptr[s + 1]; e++) {
    const int a = t.slot_ang[e];
    acc += 0.5 * (t.F[b * t.copies + 2 * a + 1] - t.F[b * t.copies + 2 * a + 2]);
  }
  grads[t.g_off + j] = (float)acc;
}

struct MultiExec final : tdq_exec {
  int dev = 0, grad = 0, nc = 0, threads = 0, fb = 0, rb = 0, grid = 0;
  std::vector<SweepExec*> subs;  // per circuit: its device tables (no kernel of its own)
  std::vector<int64_t> p_off, x_off, v_off;
  int64_t P_tot = 0, F_tot = 0, V_tot = 0, ps_total = 0;
  const void* kernel = nullptr;
  size_t smem = 0;
  MultiCirc* d_mc = nullptr;
  int2* d_items = nullptr;
  int n_items = 0;
  int* d_next = nullptr;
  int* d_status = nullptr;
  MultiPs* d_ps = nullptr;
  int last_launches = 0;
  cudaStream_t last_stream = nullptr;
  double flops_row = 0, bytes_row = 0;  // mean per row over every circuit's rows
  GraphReplay graph;

  ~MultiExec() override {
    for (SweepExec* s : subs) delete s;
    cudaFree(d_mc);
    cudaFree(d_items);
    cudaFree(d_next);
    cudaFree(d_status);
    cudaFree(d_ps);
  }

  tdq_status enqueue(const float* params, const float* inputs, double* values, const double* gw, float* grads,
                     cudaStream_t st) {
    last_launches = 0;
    TDQ_CUDA_TRY(cudaMemsetAsync(d_next, 0, sizeof(int), st));
    void* args[] = {&d_mc, &d_items, &n_items, &d_next, &params, &inputs, &values, &gw, &grads};
    TDQ_CUDA_TRY(cudaLaunchKernel(kernel, dim3(grid), dim3(threads), args, smem, st));
    last_launches++;
    if (grad == TDQ_GRAD_PARAM_SHIFT && ps_total > 0) {
      k_multi_ps_combine<<<(unsigned)((ps_total + 255) / 256), 256, 0, st>>>(d_ps, nc, ps_total, grads);
      last_launches++;
    }
    TDQ_CUDA_TRY(cudaGetLastError());
    return ok();
  }

  tdq_status execute(const float* params, int64_t pstride, const float* inputs, double* values, const double* gw,
                     float* grads, void* stream) override {
    if (!values) return fail(TDQ_ERR_ARG, "tdq_execute: values is NULL");
    if (P_tot > 0 && !params) return fail(TDQ_ERR_ARG, "tdq_execute: params is NULL");
    if (F_tot > 0 && !inputs) return fail(TDQ_ERR_ARG, "tdq_execute: inputs is NULL");
    if (pstride != 0) return fail(TDQ_ERR_ARG, "tdq_execute: a multi-circuit exec takes packed rows (params_stride 0)");
    if (grad != TDQ_GRAD_NONE && !grads) return fail(TDQ_ERR_ARG, "tdq_execute: grads is NULL");
    if (grad == TDQ_GRAD_NONE && grads)
      return fail(TDQ_ERR_ARG, "tdq_execute: grads given to an exec compiled without gradients");
    TDQ_CUDA_TRY(cudaSetDevice(dev));
    cudaStream_t st = (cudaStream_t)stream;
    last_stream = st;
    const void* key[6] = {params, inputs, values, gw, grads, stream};
    return graph.run(key, 0, st, &last_launches,
                     [&](cudaStream_t s2) { return enqueue(params, inputs, values, gw, grads, s2); });
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

  void work(double* f, double* by, int* k) const override {
    *f = flops_row;
    *by = bytes_row;
    *k = 2;
  }

  tdq_status config(int* c4) const override {
    c4[0] = threads;
    c4[1] = fb;
    c4[2] = rb;
    c4[3] = grid;
    return ok();
  }

  tdq_status multi_layout(int c, int64_t* po, int64_t* xo, int64_t* vo, int* config) const override {
    if (c < 0 || c >= nc) return fail(TDQ_ERR_ARG, "tdq_multi_layout: no such circuit");
    if (po) *po = p_off[c];
    if (xo) *xo = x_off[c];
    if (vo) *vo = v_off[c];
    if (config) {
      config[0] = threads;
      config[1] = fb;
      config[2] = rb;
      config[3] = grid;
    }
    return ok();
  }
};

// Registers per thread the multi-circuit kernel's launch bounds allow (one CTA
// of `threads` per SM), which its separately compiled row functions must keep.
static int multi_maxrreg(int threads) { return std::min(255, 65536 / threads); }

// Modules of the persistent kernel over the circuits cs (threads per CTA,
// register bits fb / rb); the same text for the export, the build and the
// autotuner, so that they share one compilation.
static std::vector<std::string> multi_modules(const tdq_circuit* const* cs, int nc, bool adj, int threads, int fb,
                                              int rb) {
  std::vector<Program> progs(nc);
  std::vector<K2Part> parts;
  for (int c = 0; c < nc; c++) {
    int npf = 0, npb = 0;
    k2_program(cs[c], adj, fb, rb, progs[c], &npf, &npb, true);
    parts.push_back({&progs[c], npf, npb, std::min(fb, cs[c]->n), std::min(rb, cs[c]->n), cs[c]->n_params, cs[c]->n});
  }
  return k2_multi_modules(parts, adj, threads, "tdq_k2_multi");
}

// One configuration of a multi-circuit launch: every circuit's tables and
// program, one kernel over all of them, the item list (costliest first).
static tdq_status multi_build(const tdq_circuit* const* cs, const int* batch, int nc, const tdq_compile_opts* o,
                              int threads, int fb, int rb, MultiExec** out) {
  *out = nullptr;
  MultiExec* e = new (std::nothrow) MultiExec();
  if (!e) return fail(TDQ_ERR_OOM, "tdq_compile_multi: host allocation");
  auto bail = [&](tdq_status s) {
    delete e;
    return s;
  };
  e->dev = o->device;
  e->grad = o->grad;
  e->nc = nc;
  e->threads = threads;
  e->fb = fb;
  e->rb = rb;
  if (cudaSetDevice(e->dev) != cudaSuccess) return bail(fail(TDQ_ERR_CUDA, "cudaSetDevice failed"));
  if (cudaMalloc(&e->d_status, sizeof(int)) != cudaSuccess || cudaMalloc(&e->d_next, sizeof(int)) != cudaSuccess)
    return bail(fail(TDQ_ERR_OOM, "tdq_compile_multi: buffers"));
  cudaMemset(e->d_status, 0, sizeof(int));
  std::vector<MultiHook> hooks(nc);
  std::vector<MultiCirc> mc(nc);
  std::vector<MultiPs> ps;
  std::vector<double> cost(nc);
  size_t smem = 0;
  for (int c = 0; c < nc; c++) {
    tdq_compile_opts oc = *o;
    oc.batch = batch[c];
    oc.fwd_reg_bits = fb;
    oc.rev_reg_bits = rb;
    oc.interpret = 0;
    hooks[c].threads = threads;
    tdq_exec* sub = nullptr;
    tdq_status s = compile_sweep_impl(cs[c], &oc, &sub, &hooks[c]);
    if (s != TDQ_OK) return bail(s);
    SweepExec* x = static_cast<SweepExec*>(sub);
    e->subs.push_back(x);
    smem = std::max(smem, x->smem_bytes);
    MultiCirc& m = mc[c];
    std::memset(&m, 0, sizeof(m));
    SweepArgs& a = m.a;
    a.ops = x->d_ops; a.G = x->G; a.n = x->n;
    a.pstride = x->P; a.F = x->F;
    a.terms = x->d_terms; a.group_ptr = x->d_group_ptr; a.T = x->T; a.n_groups = x->ng;
    a.amp_idx = x->d_amp; a.A = x->A; a.output = x->output;
    a.P = x->P; a.status = e->d_status;
    a.ps_copies = x->copies; a.ps_gate = x->d_ps_gate; a.ps_ang = x->d_ps_ang; a.ps_F = x->d_ps_F;
    a.odiag = x->d_odiag;
    m.rec_ptr = x->d_rec_ptr;
    m.rec_ops = x->d_rec_ops;
    m.nrec = x->nrec;
    m.p_off = e->P_tot;
    m.x_off = e->F_tot;
    m.v_off = e->V_tot;
    m.g_off = e->P_tot;
    e->p_off.push_back(e->P_tot);
    e->x_off.push_back(e->F_tot);
    e->v_off.push_back(e->V_tot);
    if (o->grad == TDQ_GRAD_PARAM_SHIFT && x->P > 0)
      ps.push_back({x->d_ps_F, x->d_slot_ptr, x->d_slot_ang, x->copies, x->P, e->ps_total, e->P_tot});
    e->ps_total += o->grad == TDQ_GRAD_PARAM_SHIFT ? (int64_t)batch[c] * x->P : 0;
    e->P_tot += (int64_t)batch[c] * x->P;
    e->F_tot += (int64_t)batch[c] * x->F;
    e->V_tot += (int64_t)batch[c] * x->ng;
    cost[c] = x->flops_row;  // per row, shifted copies included
    e->flops_row += x->flops_row * batch[c];
    e->bytes_row += x->bytes_row * batch[c];
  }
  int64_t rows = 0;  // work() reports the mean per row
  for (int c = 0; c < nc; c++) rows += batch[c];
  e->flops_row /= (double)rows;
  e->bytes_row /= (double)rows;
  // one kernel for all circuits
  tdq_status s = jit_link_kernel(multi_modules(cs, nc, o->grad == TDQ_GRAD_ADJOINT, threads, fb, rb), "tdq_k2_multi",
                                 multi_maxrreg(threads), &e->kernel);
  if (s != TDQ_OK) return bail(s);
  e->smem = smem;
  cudaError_t ce = cudaFuncSetAttribute(e->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (ce != cudaSuccess) return bail(fail(TDQ_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(ce)));
  // items: rows of the costliest circuits first (longest-processing-time order)
  std::vector<int> order(nc);
  for (int c = 0; c < nc; c++) order[c] = c;
  std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return cost[p] > cost[q]; });
  std::vector<int2> items;
  for (int c : order)
    for (int r = 0; r < batch[c] * e->subs[c]->copies; r++) items.push_back(make_int2(c, r));
  e->n_items = (int)items.size();
  int per_sm = 0, sms = 0;
  ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, e->kernel, threads, smem);
  if (ce != cudaSuccess || per_sm < 1)
    return bail(fail(TDQ_ERR_UNSUPPORTED, "tdq_compile_multi: the kernel does not fit an SM at this CTA size"));
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->dev);
  e->grid = (int)std::min<int64_t>(e->n_items, (int64_t)per_sm * sms);
  if ((s = upload(&e->d_mc, mc)) != TDQ_OK) return bail(s);
  if ((s = upload(&e->d_items, items)) != TDQ_OK) return bail(s);
  if ((s = upload(&e->d_ps, ps)) != TDQ_OK) return bail(s);
  if ((s = e->graph.init()) != TDQ_OK) return bail(s);
  *out = e;
  return ok();
}

// Median time (ms) of a few executions on synthetic parameters (the kernels'
// work does not depend on the values), each after an L2 flush.
static tdq_status multi_time(MultiExec* e, float* ms) {
  float* p = nullptr;
  float* x = nullptr;
  float* g = nullptr;
  double* v = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  auto done = [&](tdq_status s) {
    cudaFree(p);
    cudaFree(x);
    cudaFree(g);
    cudaFree(v);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (st) cudaStreamDestroy(st);
    return s;
  };
  const size_t np = (size_t)std::max<int64_t>(e->P_tot, 1), nx = (size_t)std::max<int64_t>(e->F_tot, 1);
  if (cudaMalloc(&p, sizeof(float) * np) != cudaSuccess || cudaMalloc(&x, sizeof(float) * nx) != cudaSuccess ||
      cudaMalloc(&g, sizeof(float) * np) != cudaSuccess ||
      cudaMalloc(&v, sizeof(double) * (size_t)std::max<int64_t>(e->V_tot, 1)) != cudaSuccess)
    return done(fail(TDQ_ERR_OOM, "tdq_compile_multi: autotune buffers"));
  std::vector<float> h(std::max(np, nx), 0.37f);
  if (cudaMemcpy(p, h.data(), sizeof(float) * np, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(x, h.data(), sizeof(float) * nx, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
      cudaEventCreate(&b) != cudaSuccess)
    return done(fail(TDQ_ERR_CUDA, "tdq_compile_multi: autotune setup"));
  float* gg = e->grad == TDQ_GRAD_NONE ? nullptr : g;
  L2Flush fl;
  tdq_status fs = fl.init(e->dev);
  if (fs != TDQ_OK) return done(fs);
  std::vector<float> t;
  for (int it = 0; it < 6; it++) {
    if (fl.run(it, st) != cudaSuccess || cudaEventRecord(a, st) != cudaSuccess)
      return done(fail(TDQ_ERR_CUDA, "tdq_compile_multi: event"));
    tdq_status s = e->enqueue(p, x, v, nullptr, gg, st);
    if (s != TDQ_OK) return done(s);
    if (cudaEventRecord(b, st) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess)
      return done(fail(TDQ_ERR_CUDA, "tdq_compile_multi: autotune run"));
    float m = 0.f;
    cudaEventElapsedTime(&m, a, b);
    if (it > 0) t.push_back(m);  // the first run warms up
  }
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  cudaMemset(e->d_status, 0, sizeof(int));
  return done(TDQ_OK);
}

}  // namespace tdq

extern "C" tdq_status tdq_compile_multi(const tdq_circuit* const* circuits, const int* batch, int n_circuits,
                                        const tdq_compile_opts* o, tdq_exec** out) {
  if (!circuits || !batch || !o || !out || n_circuits < 1) return fail(TDQ_ERR_ARG, "tdq_compile_multi: bad argument");
  *out = nullptr;
  if (o->output != TDQ_OUT_EXPVAL) return fail(TDQ_ERR_ARG, "tdq_compile_multi: expectation outputs only");
  if (o->grad < TDQ_GRAD_NONE || o->grad > TDQ_GRAD_PARAM_SHIFT)
    return fail(TDQ_ERR_ARG, "tdq_compile_multi: bad gradient mode");
  if (o->interpret) return fail(TDQ_ERR_ARG, "tdq_compile_multi: programs are always specialised (interpret = 0)");
  if (o->fwd_reg_bits < 0 || o->fwd_reg_bits > 4 || o->rev_reg_bits < 0 || o->rev_reg_bits > 4)
    return fail(TDQ_ERR_ARG, "tdq_compile_multi: register bits must be in 1..4 (0 = default)");
  if (o->autotune && (o->fwd_reg_bits || o->rev_reg_bits))
    return fail(TDQ_ERR_ARG, "tdq_compile_multi: autotune picks the register bits itself");
  const int nmax = o->grad == TDQ_GRAD_ADJOINT ? 13 : 14;
  int64_t rows = 0;
  int widest = 1;
  for (int c = 0; c < n_circuits; c++) {
    if (!circuits[c]) return fail(TDQ_ERR_ARG, "tdq_compile_multi: NULL circuit " + std::to_string(c));
    if (batch[c] < 1) return fail(TDQ_ERR_ARG, "tdq_compile_multi: batch of circuit " + std::to_string(c) + " < 1");
    if (circuits[c]->n > nmax)
      return fail(TDQ_ERR_UNSUPPORTED, "tdq_compile_multi: circuit " + std::to_string(c) + " has more than " +
                                           std::to_string(nmax) + " qubits");
    if (circuits[c]->n_groups == 0)
      return fail(TDQ_ERR_STATE, "tdq_compile_multi: circuit " + std::to_string(c) + " has no observable");
    rows += batch[c];
    widest = std::max(widest, circuits[c]->n);
  }
  if (rows > (1 << 30)) return fail(TDQ_ERR_ARG, "tdq_compile_multi: too many rows");
  MultiExec* best = nullptr;
  if (!o->autotune) {
    const int fb = o->fwd_reg_bits ? o->fwd_reg_bits : kSpecFwdRegBits;
    const int rb = o->rev_reg_bits ? o->rev_reg_bits : kSpecRevRegBits;
    const int threads = std::max(64, std::min(256, (1 << widest) >> std::min(fb, widest)));
    tdq_status s = multi_build(circuits, batch, n_circuits, o, threads, fb, rb, &best);
    if (s != TDQ_OK) return s;
  } else {
    // compile every candidate concurrently on the host's cores (NVRTC), then
    // build and time them one by one
    const std::vector<std::pair<int, int>> cands = {{128, 2}, {128, 3}, {256, 2}, {256, 3}, {512, 2}, {512, 3}};
    std::vector<tdq_status> cst(cands.size(), TDQ_OK);
    std::vector<std::string> cmsg(cands.size());
    std::vector<std::thread> pool;
    for (size_t i = 0; i < cands.size(); i++)
      pool.emplace_back([&, i] {
        try {
          if (cudaSetDevice(o->device) != cudaSuccess) {
            cst[i] = TDQ_ERR_CUDA;
            cmsg[i] = "cudaSetDevice failed";
            return;
          }
          const void* k = nullptr;
          cst[i] = jit_link_kernel(multi_modules(circuits, n_circuits, o->grad == TDQ_GRAD_ADJOINT, cands[i].first,
                                                 cands[i].second, cands[i].second),
                                   "tdq_k2_multi", multi_maxrreg(cands[i].first), &k);
          if (cst[i] != TDQ_OK) cmsg[i] = tdq_last_error();
        } catch (...) {
          cst[i] = TDQ_ERR_OOM;
          cmsg[i] = "host allocation while compiling a candidate";
        }
      });
    for (auto& t : pool) t.join();
    for (size_t i = 0; i < cands.size(); i++)
      if (cst[i] != TDQ_OK) return fail(cst[i], "tdq_compile_multi: " + cmsg[i]);
    float best_ms = 0.f;
    for (const auto& cand : cands) {
      {
        const int threads = cand.first, bits = cand.second;
        MultiExec* e = nullptr;
        tdq_status s = multi_build(circuits, batch, n_circuits, o, threads, bits, bits, &e);
        if (s == TDQ_ERR_UNSUPPORTED) continue;  // this CTA size does not fit
        if (s != TDQ_OK) {
          delete best;
          return s;
        }
        float ms = 0.f;
        s = multi_time(e, &ms);
        if (s != TDQ_OK) {
          delete e;
          delete best;
          return s;
        }
        if (!best || ms < best_ms) {
          delete best;
          best = e;
          best_ms = ms;
        } else {
          delete e;
        }
      }
    }
    if (!best) return fail(TDQ_ERR_UNSUPPORTED, "tdq_compile_multi: no launch configuration fits");
  }
  *out = best;
  return ok();
}

extern "C" tdq_status tdq_multi_source(const tdq_circuit* const* circuits, int n_circuits, int grad, int threads,
                                       int fwd_reg_bits, int rev_reg_bits, char* buf, size_t cap, size_t* len) {
  if (!circuits || n_circuits < 1 || !len) return fail(TDQ_ERR_ARG, "tdq_multi_source: bad argument");
  if (grad < TDQ_GRAD_NONE || grad > TDQ_GRAD_PARAM_SHIFT) return fail(TDQ_ERR_ARG, "tdq_multi_source: bad gradient mode");
  if (threads < 32 || threads > 1024 || threads % 32)
    return fail(TDQ_ERR_ARG, "tdq_multi_source: threads must be a multiple of 32 in 32..1024");
  if (fwd_reg_bits < 1 || fwd_reg_bits > 4 || rev_reg_bits < 1 || rev_reg_bits > 4)
    return fail(TDQ_ERR_ARG, "tdq_multi_source: register bits must be in 1..4");
  const bool adj = grad == TDQ_GRAD_ADJOINT;
  for (int c = 0; c < n_circuits; c++) {
    if (!circuits[c]) return fail(TDQ_ERR_ARG, "tdq_multi_source: NULL circuit");
    if (circuits[c]->n > (adj ? 13 : 14)) return fail(TDQ_ERR_UNSUPPORTED, "tdq_multi_source: circuit too large");
  }
  std::string src;
  const std::vector<std::string> mods = multi_modules(circuits, n_circuits, adj, threads, fwd_reg_bits, rev_reg_bits);
  for (size_t i = 0; i < mods.size(); i++) src += std::string(kModuleMark) + std::to_string(i) + "\n" + mods[i];
  *len = src.size() + 1;
  if (buf) {
    if (cap < src.size() + 1) return fail(TDQ_ERR_ARG, "tdq_multi_source: buffer too small");
    std::memcpy(buf, src.c_str(), src.size() + 1);
  }
  return ok();
}

// ------------------------------------------------- execution without allocation
//
// tdq_execute_param_shift_noalloc: the whole-state sweep with parameter-shift
// gradients for callers that cannot allocate device memory.  Every device
// table the kernels read (gate program, observable terms, shift bookkeeping)
// and the per-copy values of the shift rule live in one file-scope
// __device__ array of fixed size, shared by every call on a device.

#include <mutex>

namespace tdq {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;  // 8 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256];  // device address of the array, per device ordinal

// Device address of the scratch array for the current device, looked up once
// per device (cudaGetSymbolAddress) with that device current.
static tdq_status noalloc_scratch(int dev, unsigned char** out) {
  if (dev < 0 || dev >= 256) return fail(TDQ_ERR_ARG, "no-alloc execute: device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(TDQ_ERR_CUDA, std::string("no-alloc execute: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  return TDQ_OK;
}

}  // namespace tdq

extern "C" tdq_status tdq_execute_param_shift_noalloc(const tdq_circuit* c, int batch, const float* d_params,
                                                      int64_t params_stride, const float* d_inputs,
                                                      double* d_values, float* d_grads, void* stream) {
  if (!c) return fail(TDQ_ERR_ARG, "no-alloc execute: circuit is NULL");
  if (batch < 1) return fail(TDQ_ERR_ARG, "no-alloc execute: batch must be >= 1");
  if (c->n > 13) return fail(TDQ_ERR_ARG, "no-alloc execute: at most 13 qubits (state held in shared memory)");
  if (c->n_groups == 0) return fail(TDQ_ERR_STATE, "no-alloc execute: circuit has no observable");
  if (!d_values) return fail(TDQ_ERR_ARG, "no-alloc execute: values is NULL");
  if (c->n_params > 0 && (!d_params || !d_grads))
    return fail(TDQ_ERR_ARG, "no-alloc execute: params and grads are required");
  if (c->n_inputs > 0 && !d_inputs) return fail(TDQ_ERR_ARG, "no-alloc execute: inputs is NULL");
  if (params_stride != 0 && params_stride < c->n_params)
    return fail(TDQ_ERR_ARG, "no-alloc execute: params_stride < number of parameters");
  int dev = 0;
  TDQ_CUDA_TRY(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  tdq_status s = noalloc_scratch(dev, &base);
  if (s != TDQ_OK) return s;

  // host tables: gate program, shifted angles, terms, shift-rule bookkeeping
  const int n = c->n, G = (int)c->gates.size(), P = c->n_params, ng = c->n_groups;
  std::vector<int> ps_gate, ps_ang;
  const std::vector<SweepOp> ops = sweep_ops(c, &ps_gate, &ps_ang);
  const int NA = (int)ps_gate.size(), copies = 1 + 2 * NA;
  std::vector<TermDev> terms;
  std::vector<int> gptr(ng + 1, 0);
  for (int g = 0; g < ng; g++) {
    gptr[g] = (int)terms.size();
    for (const Term& t : c->terms) {
      if (t.group != g) continue;
      TermDev d{};
      for (int q : t.zq) d.pmask_lo |= 1u << (n - 1 - q);
      d.coeff = (float)t.coeff;
      d.group = g;
      terms.push_back(d);
    }
  }
  gptr[ng] = (int)terms.size();
  std::vector<int> sptr(P + 1, 0), sang;
  for (int sl = 0; sl < P; sl++) {
    sptr[sl] = (int)sang.size();
    for (int j = 0; j < NA; j++)
      if (ops[ps_gate[j]].slot[ps_ang[j]] == sl) sang.push_back(j);
  }
  sptr[P] = (int)sang.size();
  int8_t loc[32];
  for (int p = 0; p < 32; p++) loc[p] = (int8_t)(p < n ? p : -1);
  Program prog;
  build_program(ops, 0, G, loc, n, true, 0, kFwdRegBits, prog);

  // layout of the scratch array (16-byte aligned pieces)
  size_t used = 0;
  auto place = [&](size_t bytes) {
    const size_t at = used;
    used += (bytes + 15) & ~(size_t)15;
    return at;
  };
  const size_t o_ops = place(sizeof(SweepOp) * ops.size());
  const size_t o_terms = place(sizeof(TermDev) * terms.size());
  const size_t o_gptr = place(sizeof(int) * gptr.size());
  const size_t o_pass = place(sizeof(RegPass) * prog.passes.size());
  const size_t o_dops = place(sizeof(DOp) * prog.dops.size());
  const size_t o_rptr = place(sizeof(int) * prog.rec_ptr.size());
  const size_t o_rops = place(sizeof(int) * prog.rec_ops.size());
  const size_t o_psg = place(sizeof(int) * ps_gate.size());
  const size_t o_psa = place(sizeof(int) * ps_ang.size());
  const size_t o_sptr = place(sizeof(int) * sptr.size());
  const size_t o_sang = place(sizeof(int) * sang.size());
  const size_t o_stat = place(sizeof(int));
  const size_t tables = used;
  const size_t o_F = place(sizeof(double) * (size_t)batch * copies);
  if (used > kNoAllocScratchBytes)
    return fail(TDQ_ERR_ARG, "no-alloc execute: needs " + std::to_string(used) + " bytes of scratch, more than the " +
                                 std::to_string(kNoAllocScratchBytes) + "-byte maximum (fewer rows or angles per call)");
  std::vector<unsigned char> host(tables, 0);
  auto put = [&](size_t at, const void* src, size_t bytes) {
    if (bytes) std::memcpy(host.data() + at, src, bytes);
  };
  put(o_ops, ops.data(), sizeof(SweepOp) * ops.size());
  put(o_terms, terms.data(), sizeof(TermDev) * terms.size());
  put(o_gptr, gptr.data(), sizeof(int) * gptr.size());
  put(o_pass, prog.passes.data(), sizeof(RegPass) * prog.passes.size());
  put(o_dops, prog.dops.data(), sizeof(DOp) * prog.dops.size());
  put(o_rptr, prog.rec_ptr.data(), sizeof(int) * prog.rec_ptr.size());
  put(o_rops, prog.rec_ops.data(), sizeof(int) * prog.rec_ops.size());
  put(o_psg, ps_gate.data(), sizeof(int) * ps_gate.size());
  put(o_psa, ps_ang.data(), sizeof(int) * ps_ang.size());
  put(o_sptr, sptr.data(), sizeof(int) * sptr.size());
  put(o_sang, sang.data(), sizeof(int) * sang.size());
  cudaStream_t st = (cudaStream_t)stream;
  // the status word starts at zero (host buffer zero-filled); the per-copy
  // values are all written by the sweep kernel before the combine reads them
  TDQ_CUDA_TRY(cudaMemcpyAsync(base, host.data(), tables, cudaMemcpyHostToDevice, st));

  SweepArgs a{};
  a.ops = reinterpret_cast<const SweepOp*>(base + o_ops);
  a.G = G;
  a.n = n;
  a.params = d_params;
  a.pstride = params_stride;
  a.inputs = d_inputs;
  a.F = c->n_inputs;
  a.terms = reinterpret_cast<const TermDev*>(base + o_terms);
  a.group_ptr = reinterpret_cast<const int*>(base + o_gptr);
  a.T = (int)terms.size();
  a.n_groups = ng;
  a.amp_idx = nullptr;
  a.A = 0;
  a.output = TDQ_OUT_EXPVAL;
  a.values = d_values;
  a.gw = nullptr;
  a.grads = d_grads;
  a.P = P;
  a.status = reinterpret_cast<int*>(base + o_stat);
  a.ps_copies = copies;
  a.ps_gate = reinterpret_cast<const int*>(base + o_psg);
  a.ps_ang = reinterpret_cast<const int*>(base + o_psa);
  a.ps_F = reinterpret_cast<double*>(base + o_F);
  const int nrec = (int)prog.rec_ptr.size() - 1, ndops = (int)prog.dops.size(), npf = (int)prog.passes.size();
  const size_t smem = ((size_t)1 << n) * sizeof(c2) + sizeof(OpMat) * nrec + sizeof(DOp) * ndops +
                      32 * sizeof(double) + 16;
  if (smem > 227 * 1024) return fail(TDQ_ERR_ARG, "no-alloc execute: gate program too large for shared memory");
  const int M = std::min(kFwdRegBits, n);
  const int threads = std::max(32, std::min(kK2GenericThreads, (1 << n) >> M));
  const unsigned grid = (unsigned)((int64_t)batch * copies);
  const RegPass* dp = reinterpret_cast<const RegPass*>(base + o_pass);
  const DOp* dd = reinterpret_cast<const DOp*>(base + o_dops);
  const int* rp = reinterpret_cast<const int*>(base + o_rptr);
  const int* ro = reinterpret_cast<const int*>(base + o_rops);
  cudaError_t ce = cudaSuccess;
#define TDQ_NA(MF, MB)                                                                                     \
  do {                                                                                                     \
    ce = cudaFuncSetAttribute(k2_sweep_smem<MF, MB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                              (int)smem);                                                                  \
    if (ce == cudaSuccess)                                                                                 \
      k2_sweep_smem<MF, MB, false><<<grid, threads, smem, st>>>(a, dp, npf, 0, dd, ndops, rp, ro, nrec);    \
  } while (0)
  if (M >= 4) TDQ_NA(4, 3);
  else if (M == 3) TDQ_NA(3, 3);
  else if (M == 2) TDQ_NA(2, 2);
  else TDQ_NA(1, 1);
#undef TDQ_NA
  if (ce != cudaSuccess) return fail(TDQ_ERR_CUDA, std::string("no-alloc execute: ") + cudaGetErrorString(ce));
  const int64_t tot = (int64_t)batch * P;
  if (tot > 0)
    k_param_shift_combine<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(
        a.ps_F, copies, reinterpret_cast<const int*>(base + o_sptr), reinterpret_cast<const int*>(base + o_sang), P,
        batch, d_grads);
  TDQ_CUDA_TRY(cudaGetLastError());
  return ok();
}
