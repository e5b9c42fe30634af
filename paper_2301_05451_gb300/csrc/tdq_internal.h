// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "tdq.h"

namespace tdq {

// Records msg as the calling thread's last error and returns st.
tdq_status fail(tdq_status st, const std::string& msg);
// Clears the last error, returns TDQ_OK.
tdq_status ok();

// Number of angles each gate kind takes.
int gate_n_angles(int kind);
// 1 or 2 qubits; 0 for an unknown kind.
int gate_arity(int kind);

struct GateRec {
  int kind;
  int q[2];
  int src[3];      // >= 0 parameter column, TDQ_INPUT(j) input j, TDQ_FIXED
  double fixed[3]; // used where src == TDQ_FIXED
};

struct Term {
  std::vector<int> zq;  // qubits carrying Z
  double coeff;
  int group;
};

}  // namespace tdq

struct tdq_circuit {
  int n = 0;
  std::vector<tdq::GateRec> gates;
  std::vector<tdq::Term> terms;
  std::vector<std::vector<uint8_t>> amps;
  int n_groups = 0;
  int n_params = 0;
  int n_inputs = 0;
};

// Every exec kind implements this interface.
struct tdq_exec {
  virtual ~tdq_exec() {}
  virtual tdq_status execute(const float* params, int64_t pstride, const float* inputs,
                             double* values, const double* gw, float* grads, void* stream) = 0;
  virtual tdq_status status() = 0;
  virtual int launches() const = 0;
  virtual void work(double* flops, double* bytes, int* kclass) const = 0;
  virtual tdq_status timings(float* ms, int max, int* n) {
    (void)ms; (void)max; (void)n;
    return tdq::fail(TDQ_ERR_UNSUPPORTED, "tdq_exec_timings: not recorded by this exec kind");
  }
  virtual tdq_status set_initial_state(const float* psi0, int64_t stride) {
    (void)psi0; (void)stride;
    return tdq::fail(TDQ_ERR_UNSUPPORTED, "tdq_exec_set_initial_state: state sweeps only");
  }
  virtual tdq_status launch_work(double* flops, double* bytes, int* kind, int max, int* n) const {
    (void)flops; (void)bytes; (void)kind; (void)max; (void)n;
    return tdq::fail(TDQ_ERR_UNSUPPORTED, "tdq_exec_launch_work: tiled state sweeps only");
  }
  virtual tdq_status set_slice_range(int64_t first, int64_t count) {
    (void)first; (void)count;
    return tdq::fail(TDQ_ERR_UNSUPPORTED, "tdq_exec_set_slice_range: tree plans only");
  }
  virtual tdq_status config(int* c4) const {
    (void)c4;
    return tdq::fail(TDQ_ERR_UNSUPPORTED, "tdq_exec_config: sweeps and multi-circuit launches only");
  }
  virtual tdq_status multi_layout(int c, int64_t* p_off, int64_t* x_off, int64_t* v_off, int* config) const {
    (void)c; (void)p_off; (void)x_off; (void)v_off; (void)config;
    return tdq::fail(TDQ_ERR_UNSUPPORTED, "tdq_multi_layout: not a multi-circuit exec");
  }
};

#define TDQ_CUDA_TRY(expr)                                                            \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess)                                                            \
      return tdq::fail(TDQ_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)
