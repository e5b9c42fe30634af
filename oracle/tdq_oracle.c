/*
 * tdq_oracle.c -- the FP64 CPU oracle for the circuit tensor-network hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant with the CUDA
 * path.  Everything is the plain definition, written for readability, in
 * double precision:
 *
 *   - the gate matrices (RY printed in Sec. 3.2.1; the remaining conventions
 *     are the readings listed in the design notes: RX = exp(-i t X/2),
 *     RZ = diag(e^{-it/2}, e^{it/2}), RZZ = exp(-i t ZZ/2), U3 as in OpenQASM);
 *   - state-vector propagation |psi> = U |0...0>, applying each gate matrix to
 *     the 2^n amplitude vector in circuit order (Sec. 3.1, Eq. 1);
 *   - expectation values <psi| O |psi> of Pauli-Z products (Sec. 4, Eq. 9) and
 *     amplitudes <x|psi>;
 *   - the two-point parameter-shift rule k[f(mu+s) - f(mu-s)] with k = 1/2,
 *     s = pi/2 for exp(-i t P/2) gates (Sec. 4.2, Eq. 10);
 *   - a naive loop-nest contraction of the circuit's tensor network (Sec. 3.2.1:
 *     every gate and every |0> becomes a tensor; the expectation network appends
 *     the complex conjugate network).  Pairs are contracted in the oracle's own
 *     simple order (smallest result first); each pairwise contraction is a plain
 *     nested loop over result and summed indices.  The paper states that the
 *     order changes only the cost, not the value (Sec. 3.2.1).
 *
 * Qubit 0 is the most significant bit of the basis index (Sec. 5.1.1: the
 * zeroth qubit is written on the left).  Two-qubit gate matrices are indexed
 * 2*b(first qubit) + b(second qubit); CNOT's first qubit is the control.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double kHalfPi = 1.57079632679489661923;

/* gate kinds: the oracle's own numbering (the Python wrapper maps names) */
enum {
  OG_H = 0, OG_X = 1, OG_Y = 2, OG_Z = 3,
  OG_RX = 4, OG_RY = 5, OG_RZ = 6, OG_U3 = 7,
  OG_CNOT = 8, OG_CZ = 9, OG_RZZ = 10,
  OG_P0 = 11, OG_P1 = 12, /* projectors |0><0|, |1><1|: a wire fixed to one value (slicing, Sec. 3.2.3) */
  OG_COUNT = 13
};

int oracle_gate_arity(int kind) {
  if (kind < 0 || kind >= OG_COUNT) return -1;
  return (kind == OG_CNOT || kind == OG_CZ || kind == OG_RZZ) ? 2 : 1;
}

/* Fill m (row-major [out][in], d x d with d = 2 or 4) for one gate. */
static int gate_matrix(int kind, const double* a, cplx* m) {
  double c, s;
  switch (kind) {
    case OG_H:
      m[0] = sqrt(0.5); m[1] = sqrt(0.5); m[2] = sqrt(0.5); m[3] = -sqrt(0.5);
      return 2;
    case OG_X: m[0] = 0; m[1] = 1; m[2] = 1; m[3] = 0; return 2;
    case OG_Y: m[0] = 0; m[1] = -I; m[2] = I; m[3] = 0; return 2;
    case OG_Z: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -1; return 2;
    case OG_RX:
      c = cos(a[0] / 2); s = sin(a[0] / 2);
      m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c;
      return 2;
    case OG_RY: /* the matrix printed with the worked example of Sec. 3.2.1 */
      c = cos(a[0] / 2); s = sin(a[0] / 2);
      m[0] = c; m[1] = -s; m[2] = s; m[3] = c;
      return 2;
    case OG_RZ:
      m[0] = cexp(-I * a[0] / 2); m[1] = 0; m[2] = 0; m[3] = cexp(I * a[0] / 2);
      return 2;
    case OG_U3: /* U3(theta, phi, lambda) */
      c = cos(a[0] / 2); s = sin(a[0] / 2);
      m[0] = c;
      m[1] = -cexp(I * a[2]) * s;
      m[2] = cexp(I * a[1]) * s;
      m[3] = cexp(I * (a[1] + a[2])) * c;
      return 2;
    case OG_CNOT:
      for (int i = 0; i < 16; i++) m[i] = 0;
      m[0 * 4 + 0] = 1; m[1 * 4 + 1] = 1; m[2 * 4 + 3] = 1; m[3 * 4 + 2] = 1;
      return 4;
    case OG_CZ:
      for (int i = 0; i < 16; i++) m[i] = 0;
      m[0] = 1; m[5] = 1; m[10] = 1; m[15] = -1;
      return 4;
    case OG_RZZ:
      for (int i = 0; i < 16; i++) m[i] = 0;
      m[0] = cexp(-I * a[0] / 2); m[5] = cexp(I * a[0] / 2);
      m[10] = cexp(I * a[0] / 2); m[15] = cexp(-I * a[0] / 2);
      return 4;
    case OG_P0: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = 0; return 2;
    case OG_P1: m[0] = 0; m[1] = 0; m[2] = 0; m[3] = 1; return 2;
    default:
      return -1;
  }
}

/* Exported for the gate-convention tests: out = interleaved (re, im). */
int oracle_gate_matrix(int kind, const double* angles, double* out) {
  cplx m[16];
  int d = gate_matrix(kind, angles, m);
  if (d < 0) return -1;
  for (int i = 0; i < d * d; i++) {
    out[2 * i] = creal(m[i]);
    out[2 * i + 1] = cimag(m[i]);
  }
  return d;
}

/* ---------------------------------------------------------------- state vector */

static void apply_1q(cplx* psi, int n, int q, const cplx* m) {
  const int64_t dim = (int64_t)1 << n;
  const int64_t bit = (int64_t)1 << (n - 1 - q);
  for (int64_t x = 0; x < dim; x++) {
    if (x & bit) continue;
    cplx a0 = psi[x], a1 = psi[x | bit];
    psi[x] = m[0] * a0 + m[1] * a1;
    psi[x | bit] = m[2] * a0 + m[3] * a1;
  }
}

static void apply_2q(cplx* psi, int n, int qa, int qb, const cplx* m) {
  const int64_t dim = (int64_t)1 << n;
  const int64_t ba = (int64_t)1 << (n - 1 - qa);
  const int64_t bb = (int64_t)1 << (n - 1 - qb);
  for (int64_t x = 0; x < dim; x++) {
    if ((x & ba) || (x & bb)) continue;
    int64_t idx[4] = {x, x | bb, x | ba, x | ba | bb}; /* 2*b(qa) + b(qb) */
    cplx v[4], w[4];
    for (int i = 0; i < 4; i++) v[i] = psi[idx[i]];
    for (int r = 0; r < 4; r++) {
      w[r] = 0;
      for (int c = 0; c < 4; c++) w[r] += m[r * 4 + c] * v[c];
    }
    for (int i = 0; i < 4; i++) psi[idx[i]] = w[i];
  }
}

/* |psi> = G_{G-1} ... G_0 |psi0>, angles [G][3]; psi0 = NULL: |0...0>, else
 * 2^n (re, im) pairs (Sec. 3.1: the state vector starts from |0...0> unless
 * the user gives an initial state). */
static int run_circuit0(int n, int G, const int* kind, const int* q0, const int* q1,
                        const double* ang, const double* psi0, cplx* psi) {
  const int64_t dim = (int64_t)1 << n;
  if (psi0) {
    for (int64_t x = 0; x < dim; x++) psi[x] = psi0[2 * x] + psi0[2 * x + 1] * _Complex_I;
  } else {
    for (int64_t x = 0; x < dim; x++) psi[x] = 0;
    psi[0] = 1;
  }
  cplx m[16];
  for (int g = 0; g < G; g++) {
    int d = gate_matrix(kind[g], ang + 3 * g, m);
    if (d == 2) {
      if (q0[g] < 0 || q0[g] >= n) return -2;
      apply_1q(psi, n, q0[g], m);
    } else if (d == 4) {
      if (q0[g] < 0 || q0[g] >= n || q1[g] < 0 || q1[g] >= n || q0[g] == q1[g]) return -2;
      apply_2q(psi, n, q0[g], q1[g], m);
    } else {
      return -1;
    }
  }
  return 0;
}

static int run_circuit(int n, int G, const int* kind, const int* q0, const int* q1,
                       const double* ang, cplx* psi) {
  return run_circuit0(n, G, kind, q0, q1, ang, NULL, psi);
}

/* U |psi0> for one row (psi0 = NULL: |0...0>), as 2^n (re, im) pairs. */
int oracle_sv_state_from(int n, int G, const int* kind, const int* q0, const int* q1,
                         const double* ang, const double* psi0, double* psi_out) {
  if (n < 1 || n > 30) return -3;
  cplx* psi = (cplx*)malloc(sizeof(cplx) * ((size_t)1 << n));
  if (!psi) return -4;
  int rc = run_circuit0(n, G, kind, q0, q1, ang, psi0, psi);
  if (rc == 0) memcpy(psi_out, psi, sizeof(cplx) * ((size_t)1 << n));
  free(psi);
  return rc;
}

int oracle_sv_state(int n, int G, const int* kind, const int* q0, const int* q1,
                    const double* ang, double* psi_out) {
  if (n < 1 || n > 30) return -3;
  cplx* psi = (cplx*)malloc(sizeof(cplx) * ((size_t)1 << n));
  if (!psi) return -4;
  int rc = run_circuit(n, G, kind, q0, q1, ang, psi);
  if (rc == 0) memcpy(psi_out, psi, sizeof(cplx) * ((size_t)1 << n));
  free(psi);
  return rc;
}

/* <psi| Z_{q in mask} |psi>, zmask bit q = qubit q (not bit position). */
static double z_expectation(const cplx* psi, int n, int64_t zmask) {
  int64_t pmask = 0;
  for (int q = 0; q < n; q++)
    if ((zmask >> q) & 1) pmask |= (int64_t)1 << (n - 1 - q);
  const int64_t dim = (int64_t)1 << n;
  double acc = 0;
  for (int64_t x = 0; x < dim; x++) {
    double p = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
    acc += (__builtin_popcountll(x & pmask) & 1) ? -p : p;
  }
  return acc;
}

/* out[group] = sum_{terms t in group} coeff_t <Z_t> */
static void grouped_expvals(const cplx* psi, int n, int T, const int64_t* zmask,
                            const double* coeff, const int* group, int n_groups,
                            double* out) {
  for (int g = 0; g < n_groups; g++) out[g] = 0;
  for (int t = 0; t < T; t++) out[group[t]] += coeff[t] * z_expectation(psi, n, zmask[t]);
}

/* grouped expectations of U |psi0_b> for B rows; psi0 = NULL: |0...0>, else
 * rows of 2^n (re, im) pairs, row b at psi0 + b * 2 * psi0_stride (stride 0:
 * one state for every row). */
int oracle_expval_from(int n, int G, const int* kind, const int* q0, const int* q1,
                       int B, const double* ang, const double* psi0, int64_t psi0_stride, int T,
                       const int64_t* zmask, const double* coeff, const int* group, int n_groups,
                       double* out, int nthreads) {
  if (n < 1 || n > 30) return -3;
  for (int t = 0; t < T; t++)
    if (group[t] < 0 || group[t] >= n_groups) return -5;
  int err = 0;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
  for (int b = 0; b < B; b++) {
    cplx* psi = (cplx*)malloc(sizeof(cplx) * ((size_t)1 << n));
    if (!psi) { err = -4; continue; }
    int rc = run_circuit0(n, G, kind, q0, q1, ang + (size_t)b * G * 3,
                          psi0 ? psi0 + (size_t)b * 2 * (size_t)psi0_stride : NULL, psi);
    if (rc) err = rc;
    else grouped_expvals(psi, n, T, zmask, coeff, group, n_groups, out + (size_t)b * n_groups);
    free(psi);
  }
  return err;
}

int oracle_expval(int n, int G, const int* kind, const int* q0, const int* q1,
                  int B, const double* ang, int T, const int64_t* zmask,
                  const double* coeff, const int* group, int n_groups, double* out,
                  int nthreads) {
  if (n < 1 || n > 30) return -3;
  for (int t = 0; t < T; t++)
    if (group[t] < 0 || group[t] >= n_groups) return -5;
  int err = 0;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
  for (int b = 0; b < B; b++) {
    cplx* psi = (cplx*)malloc(sizeof(cplx) * ((size_t)1 << n));
    if (!psi) { err = -4; continue; }
    int rc = run_circuit(n, G, kind, q0, q1, ang + (size_t)b * G * 3, psi);
    if (rc) err = rc;
    else grouped_expvals(psi, n, T, zmask, coeff, group, n_groups, out + (size_t)b * n_groups);
    free(psi);
  }
  return err;
}

/* amplitudes <x_a|psi_b>; bits [A][n] with bits[a][q] the value of qubit q. */
int oracle_amplitude(int n, int G, const int* kind, const int* q0, const int* q1,
                     int B, const double* ang, int A, const uint8_t* bits, double* out,
                     int nthreads) {
  if (n < 1 || n > 30) return -3;
  int err = 0;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
  for (int b = 0; b < B; b++) {
    cplx* psi = (cplx*)malloc(sizeof(cplx) * ((size_t)1 << n));
    if (!psi) { err = -4; continue; }
    int rc = run_circuit(n, G, kind, q0, q1, ang + (size_t)b * G * 3, psi);
    if (rc) { err = rc; free(psi); continue; }
    for (int a = 0; a < A; a++) {
      int64_t x = 0;
      for (int q = 0; q < n; q++) x = (x << 1) | (bits[(size_t)a * n + q] & 1);
      out[((size_t)b * A + a) * 2] = creal(psi[x]);
      out[((size_t)b * A + a) * 2 + 1] = cimag(psi[x]);
    }
    free(psi);
  }
  return err;
}

/*
 * Parameter shift (Sec. 4.2, Eq. 10), one row of angles [G][3]: for each
 * requested (gate, angle) pair j, out[j] = 1/2 [F(a + pi/2) - F(a - pi/2)] with
 * F = sum_groups w_g f_g.  Valid for every angle of the gates here, each of
 * which enters as exp(-i a P / 2) up to a global phase.
 */
int oracle_param_shift_from(int n, int G, const int* kind, const int* q0, const int* q1,
                            const double* ang, const double* psi0, int NA, const int* which_gate,
                            const int* which_angle, int T, const int64_t* zmask,
                            const double* coeff, const int* group, int n_groups,
                            const double* w, double* out, int nthreads);

int oracle_param_shift(int n, int G, const int* kind, const int* q0, const int* q1,
                       const double* ang, int NA, const int* which_gate,
                       const int* which_angle, int T, const int64_t* zmask,
                       const double* coeff, const int* group, int n_groups,
                       const double* w, double* out, int nthreads) {
  return oracle_param_shift_from(n, G, kind, q0, q1, ang, NULL, NA, which_gate, which_angle, T, zmask,
                                 coeff, group, n_groups, w, out, nthreads);
}

/* the same from the initial state psi0 (NULL: |0...0>) */
int oracle_param_shift_from(int n, int G, const int* kind, const int* q0, const int* q1,
                            const double* ang, const double* psi0, int NA, const int* which_gate,
                            const int* which_angle, int T, const int64_t* zmask,
                            const double* coeff, const int* group, int n_groups,
                            const double* w, double* out, int nthreads) {
  if (n < 1 || n > 30) return -3;
  int err = 0;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
  for (int j = 0; j < NA; j++) {
    double* a2 = (double*)malloc(sizeof(double) * (size_t)G * 3);
    cplx* psi = (cplx*)malloc(sizeof(cplx) * ((size_t)1 << n));
    double* f = (double*)malloc(sizeof(double) * (size_t)n_groups);
    if (!a2 || !psi || !f) { err = -4; free(a2); free(psi); free(f); continue; }
    double val[2];
    for (int side = 0; side < 2; side++) {
      memcpy(a2, ang, sizeof(double) * (size_t)G * 3);
      a2[3 * which_gate[j] + which_angle[j]] += (side == 0 ? kHalfPi : -kHalfPi);
      int rc = run_circuit0(n, G, kind, q0, q1, a2, psi0, psi);
      if (rc) err = rc;
      grouped_expvals(psi, n, T, zmask, coeff, group, n_groups, f);
      val[side] = 0;
      for (int g = 0; g < n_groups; g++) val[side] += w[g] * f[g];
    }
    out[j] = 0.5 * (val[0] - val[1]);
    free(a2); free(psi); free(f);
  }
  return err;
}

/* ---------------------------------------------------------- tensor network */

typedef struct {
  int rank;
  int* labels; /* labels[0] is the most significant index of data */
  cplx* data;  /* 2^rank entries */
  int key_q, key_t; /* qubit and time of the tensor, for the linear order */
} otensor;

typedef struct {
  int count, cap;
  otensor* t;
  int next_label;
} onet;

static int net_push_key(onet* net, int rank, const int* labels, const cplx* data, int kq, int kt) {
  if (net->count == net->cap) {
    int nc = net->cap ? 2 * net->cap : 64;
    otensor* nt = (otensor*)realloc(net->t, sizeof(otensor) * (size_t)nc);
    if (!nt) return -4;
    net->t = nt;
    net->cap = nc;
  }
  otensor* t = &net->t[net->count];
  t->rank = rank;
  t->labels = (int*)malloc(sizeof(int) * (rank ? rank : 1));
  t->data = (cplx*)malloc(sizeof(cplx) * ((size_t)1 << rank));
  if (!t->labels || !t->data) return -4;
  memcpy(t->labels, labels, sizeof(int) * rank);
  memcpy(t->data, data, sizeof(cplx) * ((size_t)1 << rank));
  t->key_q = kq;
  t->key_t = kt;
  net->count++;
  return 0;
}

static void net_free(onet* net) {
  for (int i = 0; i < net->count; i++) {
    free(net->t[i].labels);
    free(net->t[i].data);
  }
  free(net->t);
  net->t = NULL;
  net->count = net->cap = 0;
}

/*
 * Append the ket network of the circuit: one |0> per qubit, one tensor per
 * gate with index order (outputs..., inputs...).  wire[q] ends as the label of
 * qubit q's open output leg.  With conj != 0 every entry is conjugated (the
 * bra network <0| U^dagger of Sec. 3.2.1) and times run backwards from tbase.
 *
 * With split != 0 a two-qubit gate whose matrix is block diagonal in its
 * first qubit, M = sum_s |s><s| (x) V_s (CNOT, CZ, RZZ), becomes two rank-3
 * tensors joined by a bond s: P[s][out][in] = [out == in == s] on the first
 * qubit and V[s][out][in] = V_s[out][in] on the second.  Summing the bond
 * gives back M exactly; it only lets the linear order cut one bond per gate.
 */
static int build_ket(onet* net, int n, int G, const int* kind, const int* q0, const int* q1,
                     const double* ang, int conj_flag, int split, int tbase, int* wire) {
  cplx zero_ket[2] = {1, 0};
  const int tdir = conj_flag ? -1 : 1;
  for (int q = 0; q < n; q++) {
    int l = net->next_label++;
    if (net_push_key(net, 1, &l, zero_ket, q, tbase - tdir)) return -4;
    wire[q] = l;
  }
  cplx m[16];
  for (int g = 0; g < G; g++) {
    int d = gate_matrix(kind[g], ang + 3 * g, m);
    if (d < 0) return -1;
    if (conj_flag)
      for (int i = 0; i < d * d; i++) m[i] = conj(m[i]);
    const int t = tbase + tdir * g;
    if (d == 2) {
      int lab[2] = {net->next_label++, wire[q0[g]]};
      if (net_push_key(net, 2, lab, m, q0[g], t)) return -4;
      wire[q0[g]] = lab[0];
      continue;
    }
    int block = 1; /* M[2a+b][2c+e] == 0 whenever a != c */
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++)
        for (int e = 0; e < 2; e++)
          if (m[(2 * a + b) * 4 + 2 * (1 - a) + e] != 0) block = 0;
    if (split && block) {
      int bond = net->next_label++;
      int la[3] = {bond, net->next_label++, wire[q0[g]]};
      int lb[3] = {bond, net->next_label++, wire[q1[g]]};
      cplx P[8], V[8];
      for (int s2 = 0; s2 < 2; s2++)
        for (int o = 0; o < 2; o++)
          for (int i = 0; i < 2; i++) {
            P[s2 * 4 + o * 2 + i] = (o == s2 && i == s2) ? 1 : 0;
            V[s2 * 4 + o * 2 + i] = m[(2 * s2 + o) * 4 + 2 * s2 + i];
          }
      if (net_push_key(net, 3, la, P, q0[g], t)) return -4;
      if (net_push_key(net, 3, lb, V, q1[g], t)) return -4;
      wire[q0[g]] = la[1];
      wire[q1[g]] = lb[1];
    } else {
      int lab[4] = {net->next_label, net->next_label + 1, wire[q0[g]], wire[q1[g]]};
      net->next_label += 2;
      /* m[out][in] == T[oa][ob][ia][ib] */
      if (net_push_key(net, 4, lab, m, q0[g] < q1[g] ? q0[g] : q1[g], t)) return -4;
      wire[q0[g]] = lab[0];
      wire[q1[g]] = lab[1];
    }
  }
  return 0;
}

static int has_label(const otensor* t, int l) {
  for (int i = 0; i < t->rank; i++)
    if (t->labels[i] == l) return 1;
  return 0;
}

/* Contract tensors a and b over every label they share: a plain loop nest. */
static int contract_pair(const otensor* A, const otensor* B, otensor* C, int64_t max_elems) {
  int shared[64], ns = 0, res[64], nr = 0;
  for (int i = 0; i < A->rank; i++) {
    if (has_label(B, A->labels[i])) shared[ns++] = A->labels[i];
    else res[nr++] = A->labels[i];
  }
  for (int i = 0; i < B->rank; i++)
    if (!has_label(A, B->labels[i])) res[nr++] = B->labels[i];
  if (nr > 40 || ((int64_t)1 << nr) > max_elems) return -6;
  C->rank = nr;
  C->labels = (int*)malloc(sizeof(int) * (nr ? nr : 1));
  C->data = (cplx*)calloc((size_t)1 << nr, sizeof(cplx));
  if (!C->labels || !C->data) return -4;
  memcpy(C->labels, res, sizeof(int) * nr);
  /* where each index of A and B takes its value from: result bit or shared bit */
  int a_from_res[64], a_pos[64], b_from_res[64], b_pos[64];
  for (int i = 0; i < A->rank; i++) {
    a_from_res[i] = 0;
    for (int j = 0; j < nr; j++)
      if (res[j] == A->labels[i]) { a_from_res[i] = 1; a_pos[i] = j; }
    if (!a_from_res[i])
      for (int j = 0; j < ns; j++)
        if (shared[j] == A->labels[i]) a_pos[i] = j;
  }
  for (int i = 0; i < B->rank; i++) {
    b_from_res[i] = 0;
    for (int j = 0; j < nr; j++)
      if (res[j] == B->labels[i]) { b_from_res[i] = 1; b_pos[i] = j; }
    if (!b_from_res[i])
      for (int j = 0; j < ns; j++)
        if (shared[j] == B->labels[i]) b_pos[i] = j;
  }
  const int64_t nres = (int64_t)1 << nr, nsum = (int64_t)1 << ns;
#pragma omp parallel for schedule(static) if (nres >= 4096)
  for (int64_t r = 0; r < nres; r++) {
    cplx acc = 0;
    for (int64_t s = 0; s < nsum; s++) {
      int64_t oa = 0, ob = 0;
      for (int i = 0; i < A->rank; i++) {
        int64_t v = a_from_res[i] ? (r >> (nr - 1 - a_pos[i])) & 1 : (s >> (ns - 1 - a_pos[i])) & 1;
        oa = (oa << 1) | v;
      }
      for (int i = 0; i < B->rank; i++) {
        int64_t v = b_from_res[i] ? (r >> (nr - 1 - b_pos[i])) & 1 : (s >> (ns - 1 - b_pos[i])) & 1;
        ob = (ob << 1) | v;
      }
      acc += A->data[oa] * B->data[ob];
    }
    C->data[r] = acc;
  }
  return 0;
}

/*
 * Contract the whole (closed) network to a scalar.  Order: repeatedly take the
 * pair of tensors that share a label and whose result has the fewest indices
 * (ties: lowest tensor positions).  peak receives the largest rank met.
 */
static int contract_all(onet* net, cplx* value, int64_t max_elems, int* peak) {
  *peak = 0;
  const int L = net->next_label;
  int* own0 = (int*)malloc(sizeof(int) * (L ? L : 1));
  int* own1 = (int*)malloc(sizeof(int) * (L ? L : 1));
  if (!own0 || !own1) { free(own0); free(own1); return -4; }
  int rc = 0;
  while (net->count > 1) {
    /* the two holders of every label (a closed network: at most two each) */
    for (int l = 0; l < L; l++) own0[l] = own1[l] = -1;
    for (int i = 0; i < net->count; i++)
      for (int k = 0; k < net->t[i].rank; k++) {
        int l = net->t[i].labels[k];
        if (own0[l] < 0) own0[l] = i; else own1[l] = i;
      }
    int bi = -1, bj = -1, best = 1 << 30;
    for (int l = 0; l < L; l++) {
      if (own0[l] < 0 || own1[l] < 0) continue;
      int i = own0[l] < own1[l] ? own0[l] : own1[l];
      int j = own0[l] < own1[l] ? own1[l] : own0[l];
      int shared = 0;
      for (int u = 0; u < net->t[i].rank; u++) shared += has_label(&net->t[j], net->t[i].labels[u]);
      int rr = net->t[i].rank + net->t[j].rank - 2 * shared;
      if (rr < best || (rr == best && (i < bi || (i == bi && j < bj)))) {
        best = rr; bi = i; bj = j;
      }
    }
    if (bi < 0) { /* disconnected pieces: outer product of the first two */
      bi = 0; bj = 1;
    }
    otensor C;
    rc = contract_pair(&net->t[bi], &net->t[bj], &C, max_elems);
    if (rc) break;
    if (C.rank > *peak) *peak = C.rank;
    free(net->t[bi].labels); free(net->t[bi].data);
    free(net->t[bj].labels); free(net->t[bj].data);
    net->t[bi] = C;
    net->t[bj] = net->t[net->count - 1];
    net->count--;
  }
  free(own0);
  free(own1);
  if (rc) return rc;
  if (net->count != 1 || net->t[0].rank != 0) return -7;
  *value = net->t[0].data[0];
  return 0;
}

/*
 * The linear order: sort tensors by (qubit, time) and fold them one by one
 * into a single accumulated tensor.  Each qubit's world line is absorbed in
 * turn, so the accumulator's open indices are the bonds crossing the cut
 * between absorbed and pending qubits.
 */
static int contract_linear(onet* net, cplx* value, int64_t max_elems, int* peak) {
  *peak = 0;
  int N = net->count;
  if (N == 0) return -7;
  int* order = (int*)malloc(sizeof(int) * N);
  for (int i = 0; i < N; i++) order[i] = i;
  for (int i = 1; i < N; i++) { /* insertion sort by (key_q, key_t, position) */
    int v = order[i], j = i - 1;
    while (j >= 0) {
      const otensor* a = &net->t[order[j]];
      const otensor* b = &net->t[v];
      int after = a->key_q > b->key_q || (a->key_q == b->key_q && a->key_t > b->key_t);
      if (!after) break;
      order[j + 1] = order[j];
      j--;
    }
    order[j + 1] = v;
  }
  otensor acc = net->t[order[0]];
  int rc = 0;
  for (int k = 1; k < N; k++) {
    otensor C;
    rc = contract_pair(&acc, &net->t[order[k]], &C, max_elems);
    if (rc) break;
    if (C.rank > *peak) *peak = C.rank;
    if (k > 1) { free(acc.labels); free(acc.data); }
    acc = C;
  }
  if (rc == 0 && acc.rank != 0) rc = -7;
  if (rc == 0) *value = acc.data[0];
  if (N > 1 && acc.data != net->t[order[0]].data) { free(acc.labels); free(acc.data); }
  free(order);
  return rc;
}

/* <x| U |0...0> by contracting the amplitude network (Sec. 3.2.1). */
int oracle_tn_amplitude(int n, int G, const int* kind, const int* q0, const int* q1,
                        const double* ang, const uint8_t* bits, double* out,
                        int64_t max_elems, int* peak_rank, int linear) {
  onet net = {0, 0, NULL, 0};
  int* wire = (int*)malloc(sizeof(int) * n);
  int rc = build_ket(&net, n, G, kind, q0, q1, ang, 0, linear, 0, wire);
  for (int q = 0; rc == 0 && q < n; q++) {
    cplx bra[2] = {bits[q] ? 0 : 1, bits[q] ? 1 : 0};
    rc = net_push_key(&net, 1, &wire[q], bra, q, G);
  }
  cplx v = 0;
  if (rc == 0) rc = linear ? contract_linear(&net, &v, max_elems, peak_rank)
                           : contract_all(&net, &v, max_elems, peak_rank);
  out[0] = creal(v);
  out[1] = cimag(v);
  net_free(&net);
  free(wire);
  return rc;
}

/* <0| U^dagger Z_mask U |0> by contracting ket, observable and conjugate bra. */
int oracle_tn_expval(int n, int G, const int* kind, const int* q0, const int* q1,
                     const double* ang, int64_t zmask, double* out, int64_t max_elems,
                     int* peak_rank, int linear) {
  onet net = {0, 0, NULL, 0};
  int* kw = (int*)malloc(sizeof(int) * n);
  int* bw = (int*)malloc(sizeof(int) * n);
  /* ket times 0..G-1, observable at G, bra times 2G..G+1 (run backwards) */
  int rc = build_ket(&net, n, G, kind, q0, q1, ang, 0, linear, 0, kw);
  if (rc == 0) rc = build_ket(&net, n, G, kind, q0, q1, ang, 1, linear, 2 * G, bw);
  for (int q = 0; rc == 0 && q < n; q++) {
    cplx op[4] = {1, 0, 0, ((zmask >> q) & 1) ? -1 : 1};
    int lab[2] = {bw[q], kw[q]};
    rc = net_push_key(&net, 2, lab, op, q, G);
  }
  cplx v = 0;
  if (rc == 0) rc = linear ? contract_linear(&net, &v, max_elems, peak_rank)
                           : contract_all(&net, &v, max_elems, peak_rank);
  out[0] = creal(v);
  out[1] = cimag(v);
  net_free(&net);
  free(kw);
  free(bw);
  return rc;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
