// K2 body: one CTA holds one row's whole state in shared memory and runs the
// forward sweep, the observable epilogue (K6) and the reverse sweep (K7) of
// the state-sweep contraction path (Sec. 3.2 (e), Sec. 4.1).
//
// The gate program is a policy: InterpProg decodes the host-built register
// passes at run time; a specialised program (generated per circuit, compiled
// at run time) has every pass and gate as straight-line code with its bits as
// compile-time constants.  Both use the same register gate kernels.
#pragma once

#include "engine.cuh"

namespace tdq {

// Gate program read from shared memory at run time.  Gradient shares go to
// FP64 shared-memory sums, one per parameter column.
struct InterpProg {
  static constexpr bool kSpecialised = false;
  const RegPass* passes;
  int npf, npb;
  const DOp* dops;  // in shared memory

  template <int MF>
  __device__ __forceinline__ void forward(c2* psi, const OpMat* mats, int dim) const {
    for (int pi = 0; pi < npf; pi++) {
      const RegPass rp = passes[pi];
      for (int grp = threadIdx.x; grp < (dim >> MF); grp += blockDim.x)
        fwd_group<MF>(psi, rp, dops, mats, 0u, (uint32_t)grp);
      __syncthreads();
    }
  }

  template <int MB>
  __device__ __forceinline__ void reverse(c2* psi, c2* lam, const OpMat* mats, int dim, double* gacc,
                                          float*) const {
    const int nbg = dim >> MB;
    for (int pi = npf + npb - 1; pi >= npf; pi--) {
      const RegPass rp = passes[pi];
      for (int g0 = 0; g0 < nbg; g0 += blockDim.x)  // uniform trip count: warp reductions inside
        adj_group<MB, true>(psi, lam, rp, dops, mats, 0u, (uint32_t)(g0 + threadIdx.x),
                            g0 + (int)threadIdx.x < nbg, gacc);
      __syncthreads();
    }
  }
};

// Shared-memory bytes of the gradient accumulators.
__host__ __device__ constexpr size_t k2_grad_bytes(bool specialised, int P, int nthreads) {
  return specialised ? sizeof(float) * (size_t)P * (size_t)(nthreads / 32) : sizeof(double) * (size_t)P;
}

// Row r of the batch (with parameter shift: sample r / copies, copy r % copies).
// layout: psi[dim] | lambda[dim] (GRAD) | mats[nrec] | dops[ndops] | grad accumulators | red[32] | bad
template <int MF, int MB, bool GRAD, class Prog>
__device__ __forceinline__ void k2_body(const SweepArgs& a, Prog prog, const DOp* gdops, int ndops,
                                        const int* rec_ptr, const int* rec_ops, int nrec, int r) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int dim = 1 << a.n;
  c2* psi = reinterpret_cast<c2*>(smem_raw);
  c2* lam = psi + dim;
  OpMat* mats = reinterpret_cast<OpMat*>(psi + (GRAD ? 2 : 1) * dim);
  DOp* dops = reinterpret_cast<DOp*>(mats + nrec);
  unsigned char* gbase = reinterpret_cast<unsigned char*>(dops + ndops);
  const size_t gbytes = GRAD ? k2_grad_bytes(Prog::kSpecialised, a.P, blockDim.x) : 0;
  double* gacc = reinterpret_cast<double*>(gbase);
  float* gpart = reinterpret_cast<float*>(gbase);
  double* red = reinterpret_cast<double*>(gbase + ((gbytes + 7) & ~(size_t)7));
  int* sbad = reinterpret_cast<int*>(red + 32);

  const int64_t b = r / a.ps_copies;
  const int k = r % a.ps_copies;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) *sbad = 0;
  __syncthreads();
  // K0: this row's gate tensors (fused products for the forward program)
  int bad = 0;
  for (int i = tid; i < nrec; i += nt) mats[i] = build_recipe(a, a.ops, rec_ptr, rec_ops, i, b, k, &bad);
  for (int i = tid; i < ndops; i += nt) dops[i] = gdops[i];
  if (bad) atomicOr(sbad, 1);
  if (a.init) {
    const c2* p0 = a.init + b * a.init_stride;
    for (int x = tid; x < dim; x += nt) psi[swz(x)] = p0[x];
  } else {
    for (int x = tid; x < dim; x += nt) psi[swz(x)] = {x == 0 ? 1.f : 0.f, 0.f};
  }
  if (GRAD) {
    if (Prog::kSpecialised)
      for (int j = tid; j < a.P * (nt >> 5); j += nt) gpart[j] = 0.f;
    else
      for (int j = tid; j < a.P; j += nt) gacc[j] = 0.0;
  }
  if (!Prog::kSpecialised) prog.dops = dops;
  __syncthreads();
  prog.template forward<MF>(psi, mats, dim);

  // observable epilogue (K6) / amplitude, state or probability read-out
  double Fval = 0.0;
  if (a.output == TDQ_OUT_EXPVAL) {
    for (int g = 0; g < a.n_groups; g++) {
      float acc = 0.f;
      const int t0 = a.group_ptr[g], t1 = a.group_ptr[g + 1];
      if (a.odiag) {
        const float* D = a.odiag + (size_t)g * dim;
        for (int x = tid; x < dim; x += nt) {
          const c2 v = psi[swz(x)];
          acc += (v.x * v.x + v.y * v.y) * D[x];
        }
      } else {
        for (int x = tid; x < dim; x += nt) {
          const c2 v = psi[swz(x)];
          acc += (v.x * v.x + v.y * v.y) * diag_weight(a.terms, t0, t1, (uint32_t)x);
        }
      }
      const double tot = block_sum((double)acc, red);
      const double w = a.gw ? a.gw[b * a.n_groups + g] : 1.0;
      Fval += w * tot;
      if (k == 0 && tid == 0) a.values[b * a.n_groups + g] = tot;
    }
  } else if (k == 0 && a.output == TDQ_OUT_AMPLITUDE) {
    for (int i = tid; i < a.A; i += nt) {
      const c2 v = psi[swz(a.amp_idx[i])];
      a.values[(b * a.A + i) * 2] = v.x;
      a.values[(b * a.A + i) * 2 + 1] = v.y;
    }
  } else if (k == 0 && a.output == TDQ_OUT_STATE) {
    for (int x = tid; x < dim; x += nt) {
      const c2 v = psi[swz(x)];
      a.values[(b * dim + x) * 2] = v.x;
      a.values[(b * dim + x) * 2 + 1] = v.y;
    }
  } else if (k == 0 && a.output == TDQ_OUT_PROBS) {
    for (int x = tid; x < dim; x += nt) {
      const c2 v = psi[swz(x)];
      a.values[b * dim + x] = (double)v.x * v.x + (double)v.y * v.y;
    }
  }
  if (a.ps_copies > 1 && tid == 0) a.ps_F[r] = Fval;

  if (GRAD) {
    // lambda = O_w psi,  O_w = sum_g w_g O_g (diagonal)
    for (int x = tid; x < dim; x += nt) {
      float d = 0.f;
      for (int g = 0; g < a.n_groups; g++) {
        const float w = a.gw ? (float)a.gw[b * a.n_groups + g] : 1.f;
        d += w * (a.odiag ? a.odiag[(size_t)g * dim + x]
                          : diag_weight(a.terms, a.group_ptr[g], a.group_ptr[g + 1], (uint32_t)x));
      }
      const c2 v = psi[swz(x)];
      lam[swz(x)] = {d * v.x, d * v.y};
    }
    __syncthreads();
    prog.template reverse<MB>(psi, lam, mats, dim, gacc, gpart);
    if (Prog::kSpecialised) {
      const int nw = nt >> 5;
      for (int j = tid; j < a.P; j += nt) {
        double s = 0.0;
        for (int w = 0; w < nw; w++) s += (double)gpart[w * a.P + j];
        a.grads[b * a.P + j] = (float)s;
      }
    } else {
      for (int j = tid; j < a.P; j += nt) a.grads[b * a.P + j] = (float)gacc[j];
    }
  }
  __syncthreads();
  if (tid == 0 && *sbad) atomicOr(a.status, 1 << TDQ_ERR_NONFINITE);
}

}  // namespace tdq
