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

// Modules of a persistent kernel `name` over several circuits: module 0 is the
// kernel, whose CTAs take (circuit, row) items (int2) from a global counter
// and call circuit c's row function (module c + 1: its specialised program);
// arguments (const MultiCirc*, const int2* items, int n_items, int* next,
// params, inputs, values, gw, grads), every buffer packed by circuit at the
// MultiCirc offsets.  grad: adjoint sweeps.  The modules compile separately
// (relocatable device code) and are linked into one kernel.
std::vector<std::string> k2_multi_modules(const std::vector<K2Part>& parts, bool grad, int nthreads,
                                          const char* name);
// Separates the modules in the one text tdq_multi_source writes: each module
// follows a line kModuleMark + its number.
constexpr const char* kModuleMark = "// ==== tdq module ";

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

// Compiles the modules concurrently (NVRTC, relocatable device code, one host
// thread each, every function within maxrreg registers -- the kernel's launch
// bounds, which separately compiled callees cannot see), links them
// (nvJitLink) and returns the kernel `name`; cached by the modules' text.
tdq_status jit_link_kernel(const std::vector<std::string>& mods, const char* name, int maxrreg, const void** kernel);

}  // namespace tdq
