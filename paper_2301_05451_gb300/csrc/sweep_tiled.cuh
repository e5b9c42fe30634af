// Kernel K1: the state sweep for states too large for one CTA's shared memory
// (14..30 qubits).  The ket tensor lives in HBM; the gate sequence is cut into
// passes.  A pass owns a set S of k bit positions (always the L lowest, so
// every tile is read in contiguous 2^L-amplitude runs); a tile is the 2^k
// amplitudes that share the bits outside S.  Each CTA loads tiles into shared
// memory, absorbs all of the pass's gates there and writes the tile back:
// one HBM read and write of the state per pass instead of one per gate.
// Gates acting on bits outside S are still absorbed when those bits are
// constant on the tile: diagonal gates (RZ, Z, CZ, RZZ) and CNOT controls.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "engine.cuh"
#include "sweep_common.cuh"
#include "tdq_internal.h"

namespace tdq {

struct SweepArgs;

// Algorithmic FP32 work of one gate on a state of dim amplitudes, by the
// counting rule of the design notes: a dense 2x2 complex gate 28 flops per
// amplitude pair, a diagonal phase 6 per amplitude, permutations and sign
// flips (CNOT, CZ) none; the gradient dot products of its angles.
inline double gate_fwd_flops(int kind, double dim) {
  switch (kind) {
    case K_CNOT: case K_CZ: return 0.0;
    case K_RZ: case K_Z: case K_RZZ: return 6 * dim;
    default: return 28 * dim / 2;
  }
}
inline double gate_dot_flops(int kind, double dim) {
  if (kind == K_RX || kind == K_RY) return 8 * dim / 2;
  if (kind == K_RZ || kind == K_RZZ) return 4 * dim;
  if (kind == K_U3) return (4 + 28 + 8 + 4) * dim / 2;
  return 0.0;
}

struct TiledPass {
  uint32_t smask;  // bit positions held in the tile
  int op_begin, op_end;
};

struct TiledSweep {
  int n = 0, k = 0, L = 0;
  int rows = 0;        // rows (batch x shift copies) per execute
  int chunk_rows = 0;  // rows resident at once
  bool adj = false;
  int P = 0, ng = 0;
  std::vector<TiledPass> passes;
  SweepOp* d_ops = nullptr;  // ops in pass order
  int* d_off = nullptr;      // per pass: 2^(k-L) offsets of the high tile bits
  int8_t* d_loc = nullptr;   // per pass: 32 entries, local bit of a position or -1
  c2* d_psi = nullptr;
  c2* d_lam = nullptr;
  double* d_gacc = nullptr;  // [chunk_rows][P]
  double* d_vals = nullptr;  // [chunk_rows][ng]
  int max_pass_ops = 0;
  std::vector<int> order;         // circuit gate index of each pass-ordered op
  int* d_ps_gate_pass = nullptr;  // shifted gates renumbered to pass order
  RegPass* d_rpass = nullptr;     // register passes of every tile pass
  DOp* d_dops = nullptr;
  int* d_rec_ptr = nullptr;
  int* d_rec_ops = nullptr;
  // per tile pass: forward / reverse register passes, recipe range, reverse ops
  std::vector<int> fp_begin, fp_end, bp_begin, bp_end, rec_begin, rec_end, bo_begin, bo_end;
  std::vector<int> dop_begin, dop_end;
  int max_rec = 0, max_dops = 0;
  // specialised programs (empty: interpreted): kernels per tile pass and the
  // shared-memory bytes of each pass's gradient rows
  std::vector<const void*> kf, kr;
  std::vector<int> spec_gbytes;
  int nthreads = 256, nthreads_r = 256;  // forward / reverse kernels
  std::vector<size_t> smem_f;            // per forward kernel
  size_t smem_r = 0;
  int dbl = 1;                           // double-buffered tile loads
  int fb = 4, rb = 3;                    // register bits of forward / reverse passes
  std::vector<int> slots_f;              // resident CTAs of each forward kernel on the GPU
  int slots_r = 1;                       // ... of the reverse kernels
  // launch units of one chunk, in launch order (forward passes, then reverse
  // passes last to first): algorithmic FLOPs and bytes per row, kind
  // (0 forward, 1 fused last pass, 2 reverse)
  std::vector<double> unit_flops, unit_bytes;
  std::vector<int> unit_kind;
  std::vector<cudaEvent_t> ev;  // with timings: start / end of every unit of the first chunk
};

// A decoded gate program: register passes over decoded ops, and the recipes
// of the per-row gate-tensor table the ops index.
struct Program {
  std::vector<RegPass> passes;
  std::vector<DOp> dops;
  std::vector<int> rec_ptr{0};
  std::vector<int> rec_ops;
};

// Append to P the program of ops [b, e): register passes of min(mreg, k) tile
// bits (loc maps a global position to its tile bit, -1 outside the tile).
// fuse: one-qubit gates on the same qubit within a pass share one product
// tensor (forward programs; reverse programs keep one op per gate for the
// gradients).  rec0: recipe numbering starts at P's recipe count minus rec0.
void build_program(const std::vector<SweepOp>& ops, int b, int e, const int8_t* loc, int k, bool fuse,
                   int rec0, int mreg, Program& P);


void tiled_free(TiledSweep& t);
// Host side of a tiled plan: the pass-ordered ops, per-pass high-bit offsets
// and local-bit maps, the decoded program, shifted gates in pass order.
struct TiledHost {
  std::vector<SweepOp> pops;
  std::vector<int> offs;
  std::vector<int8_t> locs;
  Program prog;
  std::vector<int> psp;
};

// The pass schedule and programs of t (host only, no device call).
// fb / rb: register bits of forward / reverse register passes.
tdq_status tiled_plan(TiledSweep& t, const tdq_circuit* c, const std::vector<SweepOp>& ops,
                      const std::vector<int>& ps_gate, int rows, bool adj, int tile_qubits, int fb, int rb,
                      TiledHost& h);

tdq_status tiled_compile(TiledSweep& t, const tdq_circuit* c, const std::vector<SweepOp>& ops,
                         const std::vector<int>& ps_gate, int rows, bool adj, int tile_qubits, bool interpret,
                         int fb, int rb, double* bytes_row);
tdq_status tiled_execute(TiledSweep& t, const SweepArgs& a, int grad, cudaStream_t st,
                         int* launches);

}  // namespace tdq
