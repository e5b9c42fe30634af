// Circuit IR (the QInterpreter's record of a quantum function, Sec. 2) and
// the small error/version entry points of the C ABI.
#include <cmath>
#include <new>
#include <string>

#include "tdq_internal.h"

namespace tdq {

static thread_local std::string g_last_error;

tdq_status fail(tdq_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

tdq_status ok() {
  g_last_error.clear();
  return TDQ_OK;
}

int gate_n_angles(int kind) {
  switch (kind) {
    case TDQ_RX: case TDQ_RY: case TDQ_RZ: case TDQ_RZZ: return 1;
    case TDQ_U3: return 3;
    default: return 0;
  }
}

int gate_arity(int kind) {
  if (kind >= TDQ_H && kind <= TDQ_U3) return 1;
  if (kind >= TDQ_CNOT && kind <= TDQ_RZZ) return 2;
  return 0;
}

}  // namespace tdq

using namespace tdq;

extern "C" {

const char* tdq_last_error(void) { return g_last_error.c_str(); }

int tdq_version(void) { return 100; }

tdq_status tdq_circuit_create(int n_qubits, tdq_circuit** out) {
  if (!out) return fail(TDQ_ERR_ARG, "tdq_circuit_create: out is NULL");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > 64)
    return fail(TDQ_ERR_ARG, "tdq_circuit_create: n_qubits must be in 1..64");
  tdq_circuit* c = new (std::nothrow) tdq_circuit();
  if (!c) return fail(TDQ_ERR_OOM, "tdq_circuit_create: out of host memory");
  c->n = n_qubits;
  *out = c;
  return ok();
}

tdq_status tdq_circuit_gate(tdq_circuit* c, int kind, const int* qubits, int nq,
                            const int* angle_src, const double* fixed) {
  if (!c) return fail(TDQ_ERR_ARG, "tdq_circuit_gate: circuit is NULL");
  const int ar = gate_arity(kind);
  if (ar == 0) return fail(TDQ_ERR_ARG, "tdq_circuit_gate: unknown gate kind " + std::to_string(kind));
  if (nq != ar || !qubits)
    return fail(TDQ_ERR_ARG, "tdq_circuit_gate: gate needs " + std::to_string(ar) + " qubits");
  GateRec g{};
  g.kind = kind;
  g.q[1] = -1;
  for (int i = 0; i < nq; i++) {
    if (qubits[i] < 0 || qubits[i] >= c->n)
      return fail(TDQ_ERR_ARG, "tdq_circuit_gate: qubit out of range");
    g.q[i] = qubits[i];
  }
  if (nq == 2 && g.q[0] == g.q[1]) return fail(TDQ_ERR_ARG, "tdq_circuit_gate: repeated qubit");
  const int na = gate_n_angles(kind);
  for (int i = 0; i < 3; i++) {
    g.src[i] = TDQ_FIXED;
    g.fixed[i] = 0.0;
  }
  if (na > 0 && !angle_src) return fail(TDQ_ERR_ARG, "tdq_circuit_gate: angle_src is NULL");
  for (int i = 0; i < na; i++) {
    const int s = angle_src[i];
    if (s == TDQ_FIXED) {
      if (!fixed) return fail(TDQ_ERR_ARG, "tdq_circuit_gate: fixed angle without `fixed`");
      if (!std::isfinite(fixed[i])) return fail(TDQ_ERR_NONFINITE, "tdq_circuit_gate: fixed angle");
      g.fixed[i] = fixed[i];
    } else if (s >= 0) {
      if (s >= (1 << 20)) return fail(TDQ_ERR_ARG, "tdq_circuit_gate: parameter column too large");
      if (s + 1 > c->n_params) c->n_params = s + 1;
    } else {
      const int j = -2 - s;
      if (j < 0 || j >= (1 << 20)) return fail(TDQ_ERR_ARG, "tdq_circuit_gate: bad input index");
      if (j + 1 > c->n_inputs) c->n_inputs = j + 1;
    }
    g.src[i] = s;
  }
  c->gates.push_back(g);
  return ok();
}

tdq_status tdq_circuit_observable(tdq_circuit* c, const int* z_qubits, int nz, double coeff,
                                  int group) {
  if (!c) return fail(TDQ_ERR_ARG, "tdq_circuit_observable: circuit is NULL");
  if (nz < 0 || (nz > 0 && !z_qubits) || group < 0 || group >= (1 << 16))
    return fail(TDQ_ERR_ARG, "tdq_circuit_observable: bad arguments");
  if (!std::isfinite(coeff)) return fail(TDQ_ERR_NONFINITE, "tdq_circuit_observable: coeff");
  Term t;
  t.coeff = coeff;
  t.group = group;
  for (int i = 0; i < nz; i++) {
    if (z_qubits[i] < 0 || z_qubits[i] >= c->n)
      return fail(TDQ_ERR_ARG, "tdq_circuit_observable: qubit out of range");
    for (int q : t.zq)
      if (q == z_qubits[i]) return fail(TDQ_ERR_ARG, "tdq_circuit_observable: repeated qubit");
    t.zq.push_back(z_qubits[i]);
  }
  c->terms.push_back(t);
  if (group + 1 > c->n_groups) c->n_groups = group + 1;
  return ok();
}

tdq_status tdq_circuit_amplitude(tdq_circuit* c, const uint8_t* bits) {
  if (!c || !bits) return fail(TDQ_ERR_ARG, "tdq_circuit_amplitude: NULL argument");
  std::vector<uint8_t> b(c->n);
  for (int q = 0; q < c->n; q++) {
    if (bits[q] > 1) return fail(TDQ_ERR_ARG, "tdq_circuit_amplitude: bits must be 0 or 1");
    b[q] = bits[q];
  }
  c->amps.push_back(b);
  return ok();
}

tdq_status tdq_circuit_info(const tdq_circuit* c, int* n_gates, int* n_params, int* n_inputs,
                            int* n_groups, int* n_terms, int* n_amplitudes) {
  if (!c) return fail(TDQ_ERR_ARG, "tdq_circuit_info: circuit is NULL");
  if (n_gates) *n_gates = (int)c->gates.size();
  if (n_params) *n_params = c->n_params;
  if (n_inputs) *n_inputs = c->n_inputs;
  if (n_groups) *n_groups = c->n_groups;
  if (n_terms) *n_terms = (int)c->terms.size();
  if (n_amplitudes) *n_amplitudes = (int)c->amps.size();
  return ok();
}

tdq_status tdq_circuit_destroy(tdq_circuit* c) {
  delete c;
  return ok();
}

tdq_status tdq_execute(tdq_exec* e, const float* d_params, int64_t params_stride,
                       const float* d_inputs, double* d_values, const double* d_grad_w,
                       float* d_grads, void* stream) {
  if (!e) return fail(TDQ_ERR_ARG, "tdq_execute: exec is NULL");
  return e->execute(d_params, params_stride, d_inputs, d_values, d_grad_w, d_grads, stream);
}

tdq_status tdq_exec_status(tdq_exec* e) {
  if (!e) return fail(TDQ_ERR_ARG, "tdq_exec_status: exec is NULL");
  return e->status();
}

int tdq_exec_launches(const tdq_exec* e) { return e ? e->launches() : -1; }

tdq_status tdq_exec_work(const tdq_exec* e, double* flops_per_row, double* bytes_per_row,
                         int* kernel_class) {
  if (!e) return fail(TDQ_ERR_ARG, "tdq_exec_work: exec is NULL");
  double f = 0, b = 0;
  int k = 0;
  e->work(&f, &b, &k);
  if (flops_per_row) *flops_per_row = f;
  if (bytes_per_row) *bytes_per_row = b;
  if (kernel_class) *kernel_class = k;
  return ok();
}

tdq_status tdq_exec_timings(tdq_exec* e, float* ms, int max, int* n) {
  if (!e) return fail(TDQ_ERR_ARG, "tdq_exec_timings: exec is NULL");
  return e->timings(ms, max, n);
}

tdq_status tdq_exec_launch_work(const tdq_exec* e, double* flops, double* bytes, int* kind, int max, int* n) {
  if (!e) return fail(TDQ_ERR_ARG, "tdq_exec_launch_work: exec is NULL");
  return e->launch_work(flops, bytes, kind, max, n);
}

tdq_status tdq_exec_config(const tdq_exec* e, int* config) {
  if (!e || !config) return fail(TDQ_ERR_ARG, "tdq_exec_config: NULL argument");
  return e->config(config);
}

tdq_status tdq_multi_layout(const tdq_exec* e, int c, int64_t* params_off, int64_t* inputs_off, int64_t* values_off,
                            int* config) {
  if (!e) return fail(TDQ_ERR_ARG, "tdq_multi_layout: exec is NULL");
  return e->multi_layout(c, params_off, inputs_off, values_off, config);
}

tdq_status tdq_exec_set_slice_range(tdq_exec* e, int64_t first, int64_t count) {
  if (!e) return fail(TDQ_ERR_ARG, "tdq_exec_set_slice_range: exec is NULL");
  return e->set_slice_range(first, count);
}

tdq_status tdq_exec_set_initial_state(tdq_exec* e, const float* d_psi0, int64_t row_stride) {
  if (!e) return fail(TDQ_ERR_ARG, "tdq_exec_set_initial_state: exec is NULL");
  return e->set_initial_state(d_psi0, row_stride);
}

tdq_status tdq_exec_destroy(tdq_exec* e) {
  delete e;
  return ok();
}

}  // extern "C"
