// Specialised sweep programs: the register passes of one circuit written out
// as straight-line device code (every gate kind, register bit and table row a
// compile-time constant), compiled at run time for the device in use.
#pragma once

#include <string>
#include <vector>

#include "sweep_tiled.cuh"
#include "tdq_internal.h"

namespace tdq {

// Source of a K2 kernel named `name` for the program `prog` of an n-qubit
// state: forward passes [0, npf), reverse passes [npf, npf + npb) (npb = 0:
// no gradients).  mf / mb register bits, nthreads threads per CTA, P gradient
// columns.
std::string k2_specialised_source(const Program& prog, int npf, int npb, int mf, int mb, int nthreads,
                                  int P, int n, const char* name);

// One circuit of a multi-circuit whole-state kernel.
struct K2Part {
  const Program* prog;
  int npf, npb, mf, mb, P, n;
};

// Source of a persistent kernel `name` over several circuits: CTAs take
// (circuit, row) items (int2) from a global counter and run that circuit's
// specialised program on that row; arguments (const MultiCirc*, const int2*
// items, int n_items, int* next, params, inputs, values, gw, grads), every
// buffer packed by circuit at the MultiCirc offsets.  grad: adjoint sweeps.
std::string k2_multi_source(const std::vector<K2Part>& parts, bool grad, int nthreads, const char* name);

// Source of the K1 kernels of every tile pass p of t (program prog):
// tdq_k1f_<p> (forward; the last one also runs its reverse sweep with
// gradients) and tdq_k1r_<p> (reverse, passes before the last).  nacc[p]:
// gradient accumulators of pass p (per-warp FP32 rows in shared memory).
std::string k1_specialised_source(const TiledSweep& t, const Program& prog, int nthreads, int nthreads_r,
                                  std::vector<int>* nacc);

// Compiles `src` for the current device and returns the kernel `name` (a
// handle usable with cudaLaunchKernel / cudaFuncSetAttribute).  Compiled
// kernels are cached by source for the life of the process.
tdq_status jit_kernel(const std::string& src, const char* name, const void** kernel);

}  // namespace tdq
