// Specialised sweep programs: the register passes of one circuit written out
// as straight-line device code (every gate kind, register bit and table row a
// compile-time constant), compiled at run time for the device in use.
#pragma once

#include <string>
#include <vector>

#include "sweep_tiled.cuh"
#include "tdq_internal.h"

namespace tdq {

// Source of a K2 kernel named `name` for the program `prog`: forward passes
// [0, npf), reverse passes [npf, npf + npb) (npb = 0: no gradients).  mf / mb
// register bits, nthreads threads per CTA, P gradient columns.
std::string k2_specialised_source(const Program& prog, int npf, int npb, int mf, int mb, int nthreads,
                                  int P, const char* name);

// Compiles `src` for the current device and returns the kernel `name` (a
// handle usable with cudaLaunchKernel / cudaFuncSetAttribute).  Compiled
// kernels are cached by source for the life of the process.
tdq_status jit_kernel(const std::string& src, const char* name, const void** kernel);

}  // namespace tdq
