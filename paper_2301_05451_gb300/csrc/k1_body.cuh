// K1 bodies: the tiled state sweep through HBM (one launch per tile pass).
// A pass holds k bit positions of the state (always the L lowest, so tiles
// are read in contiguous 2^L-amplitude runs); a tile is the 2^k amplitudes
// that share the bits outside them.  Each CTA loads its tiles into shared
// memory, absorbs the pass's gates there (register passes) and writes them
// back: one HBM read and write of the state per pass instead of one per gate.
//
// The gate program of a pass is a policy, as for K2: InterpTile decodes the
// host-built register passes at run time; a specialised program has them as
// straight-line code (bits, kinds and table rows compile-time constants).
#pragma once

#include "engine.cuh"

namespace tdq {

struct TiledDev {
  const SweepOp* ops;
  const int* off;      // this pass's 2^(k-L) offsets
  const int8_t* loc;   // this pass's 32 local-bit entries
  const RegPass* fp;   // this pass's forward register passes (ops relative to dop0)
  int nfp;
  const RegPass* bp;   // reverse register passes
  int nbp;
  const DOp* dops;     // this pass's decoded ops (forward then reverse)
  int ndops;
  int bo0, bo1;        // reverse ops range (relative)
  const int* rec_ptr;
  const int* rec_ops;
  int rec0, nrec;      // this pass's recipes
  c2* psi;
  c2* lam;
  double* gacc;
  double* vals;
  int n, k, L;
  uint32_t smask;
  int op_begin, op_end;
  int tiles_per_cta, ntiles;  // (tiles_per_cta: (row, tile) units per CTA)
  int row0;
  int nrows;           // rows of the chunk: units are (row, tile), row-major
  int gbytes;          // shared-memory bytes of the gradient partial sums
  int dbl;             // 1: two tile buffers per state (loads overlap compute)
};

// Spread the bits of t over the positions of mask (lowest first).
__device__ __forceinline__ uint32_t deposit(uint32_t t, uint32_t mask) {
  uint32_t out = 0;
  for (uint32_t m = mask; m && t; m &= m - 1, t >>= 1)
    if (t & 1u) out |= m & (0u - m);
  return out;
}

struct TileShared {
  c2* psi;
  c2* lam;
  c2* psi2;     // second buffers (double-buffered loads), or NULL
  c2* lam2;
  OpMat* mats;  // [recipes of the pass]
  DOp* dops;    // [decoded ops of the pass]
  double* red;
  double* vsum;         // [n_groups]
  unsigned char* gpart; // gradient partial sums (policy-defined), gbytes
  int* off;
  int8_t* loc;
};

// layout: psi[2^k] x npsi | lambda[2^k] x nlam | mats[nrec] | dops[ndops] | red[32] |
//         vsum[ng] | gpart[gbytes] | off[2^(k-L)] | loc[32]
__host__ __device__ __forceinline__ size_t k1_smem_bytes(int k, int L, int npsi, int nlam, int nrec, int ndops,
                                                        int ng, int gbytes) {
  return (size_t)(1 << k) * sizeof(c2) * (npsi + nlam) + sizeof(OpMat) * nrec + sizeof(DOp) * ndops +
         (32 + (size_t)ng) * sizeof(double) + (((size_t)gbytes + 7) & ~(size_t)7) + sizeof(int) * (1 << (k - L)) +
         32 + 16;
}

__device__ __forceinline__ TileShared carve(unsigned char* raw, int k, int L, int npsi, int nlam, int nrec,
                                            int ndops, int ng, int gbytes) {
  TileShared s;
  const int nloc = 1 << k;
  c2* p = reinterpret_cast<c2*>(raw);
  s.psi = p;
  s.psi2 = npsi > 1 ? p + nloc : nullptr;
  p += npsi * nloc;
  s.lam = nlam > 0 ? p : nullptr;
  s.lam2 = nlam > 1 ? p + nloc : nullptr;
  p += nlam * nloc;
  s.mats = reinterpret_cast<OpMat*>(p);
  s.dops = reinterpret_cast<DOp*>(s.mats + nrec);
  s.red = reinterpret_cast<double*>(s.dops + ndops);
  s.vsum = s.red + 32;
  s.gpart = reinterpret_cast<unsigned char*>(s.vsum + ng);
  s.off = reinterpret_cast<int*>(s.gpart + ((gbytes + 7) & ~7));
  s.loc = reinterpret_cast<int8_t*>(s.off + (1 << (k - L)));
  return s;
}

__device__ __forceinline__ uint32_t gidx(const TileShared& s, uint32_t base, uint32_t j, int L) {
  return base + (uint32_t)s.off[j >> L] + (j & ((1u << L) - 1u));
}

// Diagonal weight of output group g at basis index x: from the table of
// every group's diagonal when the compile made one (read through L2, the
// same for every row), else from the group's Z-product terms.
__device__ __forceinline__ float obs_weight(const SweepArgs& a, int g, uint32_t x) {
  if (a.odiag) return a.odiag[((size_t)g << a.n) + x];
  return diag_weight(a.terms, a.group_ptr[g], a.group_ptr[g + 1], x);
}

// Per-CTA set-up: offsets, local bits, this row's gate tensors (K0), the
// decoded ops (interpreted programs) and zeroed partial sums.
__device__ __forceinline__ void k1_setup(const SweepArgs& a, const TiledDev& t, const TileShared& s, int64_t b,
                                         int kk, int* bad) {
  const int noff = 1 << (t.k - t.L);
  for (int i = threadIdx.x; i < noff; i += blockDim.x) s.off[i] = t.off[i];
  if (threadIdx.x < 32) s.loc[threadIdx.x] = t.loc[threadIdx.x];
  // shifted gates are numbered in pass order (tiled_compile)
  for (int i = threadIdx.x; i < t.nrec; i += blockDim.x)
    s.mats[i] = build_recipe(a, t.ops, t.rec_ptr, t.rec_ops, t.rec0 + i, b, kk, bad);
  for (int i = threadIdx.x; i < t.ndops; i += blockDim.x) s.dops[i] = t.dops[i];
  for (int i = threadIdx.x; i < t.gbytes / 4; i += blockDim.x) reinterpret_cast<float*>(s.gpart)[i] = 0.f;
  for (int g = threadIdx.x; g < a.n_groups; g += blockDim.x) s.vsum[g] = 0.0;
  __syncthreads();
}

// Gate program decoded at run time; gradient shares in FP64 per (recipe, angle).
struct InterpTile {
  __device__ __forceinline__ static void forward(const TiledDev& t, const TileShared& s, uint32_t base) {
    const int ngroups = 1 << (t.k - kFwdRegBits);
    for (int i = 0; i < t.nfp; i++) {
      const RegPass rp = t.fp[i];
      for (int grp = threadIdx.x; grp < ngroups; grp += blockDim.x)
        fwd_group<kFwdRegBits>(s.psi, rp, s.dops, s.mats, base, (uint32_t)grp);
      __syncthreads();
    }
  }
  __device__ __forceinline__ static void reverse(const TiledDev& t, const TileShared& s, uint32_t base) {
    const int ngroups = 1 << (t.k - kRevRegBits);
    double* gp = reinterpret_cast<double*>(s.gpart);
    for (int i = t.nbp - 1; i >= 0; i--) {
      const RegPass rp = t.bp[i];
      for (int g0 = 0; g0 < ngroups; g0 += blockDim.x)
        adj_group<kRevRegBits, false>(s.psi, s.lam, rp, s.dops, s.mats, base, (uint32_t)(g0 + threadIdx.x),
                                         g0 + (int)threadIdx.x < ngroups, gp);
      __syncthreads();
    }
  }
  // partial sums into the row's gradient columns
  __device__ __forceinline__ static void flush(const SweepArgs& a, const TiledDev& t, const TileShared& s, int lr) {
    __syncthreads();
    const double* gp = reinterpret_cast<const double*>(s.gpart);
    for (int i = t.bo0 + (int)threadIdx.x; i < t.bo1; i += blockDim.x) {
      const DOp d = s.dops[i];
      for (int j = 0; j < d.nang; j++)
        if (d.slot[j] >= 0) atomicAdd(&t.gacc[(int64_t)lr * a.P + d.slot[j]], gp[3 * d.mat + j]);
    }
  }
};

// Starts the asynchronous load of tile `base` of state g into buffer buf
// (one commit group per thread).
__device__ __forceinline__ void k1_issue(c2* buf, const c2* g, const TileShared& s, uint32_t base, int k, int L) {
  for (uint32_t j = threadIdx.x; j < (1u << k); j += blockDim.x) cp_async8(&buf[swz(j)], &g[gidx(s, base, j, L)]);
}

// The (row, tile) units of this CTA: a contiguous range of the row-major
// unit index, cut into per-row segments; f(lr, tile0, tile1) runs one.
template <class F>
__device__ __forceinline__ void k1_for_segments(const TiledDev& t, F&& f) {
  const int64_t total = (int64_t)t.nrows * t.ntiles;
  int64_t u = (int64_t)blockIdx.x * t.tiles_per_cta;
  const int64_t u1 = min(total, u + t.tiles_per_cta);
  bool first = true;
  while (u < u1) {
    const int lr = (int)(u / t.ntiles);
    const int tile0 = (int)(u - (int64_t)lr * t.ntiles);
    const int tile1 = (int)min((int64_t)t.ntiles, tile0 + (u1 - u));
    if (!first) __syncthreads();  // the previous row's partial sums are read out
    f(lr, tile0, tile1);
    first = false;
    u += tile1 - tile0;
  }
}

// Forward pass.  FIRST: the tile starts as the initial state (|0...0> or the
// caller's) instead of being read.  LAST: accumulate the observable groups; with GRAD also form lambda = O_w psi
// and run this pass's reverse sweep at once (psi and lambda then written).
// Tiles after the first of a row segment are read while the previous one is
// being computed (two shared-memory buffers).
template <bool FIRST, bool LAST, bool GRAD, class Prog>
__device__ __forceinline__ void k1_forward_body(const SweepArgs& a, const TiledDev& t, int store) {
  extern __shared__ __align__(16) unsigned char raw[];
  const TileShared s = carve(raw, t.k, t.L, (FIRST || !t.dbl) ? 1 : 2, (GRAD && LAST) ? 1 : 0, t.nrec, t.ndops,
                             a.n_groups, t.gbytes);
  const uint32_t nloc = 1u << t.k;
  const uint32_t dim = 1u << t.n;
  const uint32_t other = (dim - 1u) & ~t.smask;
  k1_for_segments(t, [&](int lr, int tile0, int tile1) {
    const int row = t.row0 + lr;
    const int64_t b = row / a.ps_copies;
    const int kk = row % a.ps_copies;
    int bad = 0;
    k1_setup(a, t, s, b, kk, &bad);
    if (bad) atomicOr(a.status, 1 << TDQ_ERR_NONFINITE);
    c2* gpsi = t.psi + (size_t)lr * dim;
    c2* glam = GRAD ? t.lam + (size_t)lr * dim : nullptr;
    if (!FIRST && t.dbl && tile0 < tile1) {
      k1_issue(s.psi, gpsi, s, deposit((uint32_t)tile0, other), t.k, t.L);
      cp_async_commit();
    }
    for (int tile = tile0, it = 0; tile < tile1; tile++, it++) {
      const uint32_t base = deposit((uint32_t)tile, other);
      TileShared sc = s;
      if (FIRST && !a.init && base != 0u) {
        // from |0...0>, the pass's gates mix amplitudes within a tile only,
        // so every tile but the one at base 0 stays zero: write it out as
        // zeros (psi, and lambda = O psi = 0 when the reverse sweep is fused)
        // without its gates; nothing in shared memory is touched
        if (store || (LAST && GRAD))
          for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) {
            const uint32_t x = gidx(s, base, j, t.L);
            gpsi[x] = {0.f, 0.f};
            if (LAST && GRAD) glam[x] = {0.f, 0.f};
          }
        continue;
      }
      if (FIRST) {
        if (a.init) {
          const c2* p0 = a.init + b * a.init_stride;
          for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) sc.psi[swz(j)] = p0[gidx(s, base, j, t.L)];
        } else {
          for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x)
            sc.psi[swz(j)] = {(base == 0u && j == 0u) ? 1.f : 0.f, 0.f};
        }
      } else if (t.dbl) {
        sc.psi = (it & 1) ? s.psi2 : s.psi;
        if (tile + 1 < tile1) {  // the buffer of the previous tile is free (barrier at the loop end)
          k1_issue((it & 1) ? s.psi : s.psi2, gpsi, s, deposit((uint32_t)(tile + 1), other), t.k, t.L);
          cp_async_commit();
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
      } else {  // one buffer: load, then compute
        k1_issue(s.psi, gpsi, s, base, t.k, t.L);
        cp_async_commit();
        cp_async_wait<0>();
      }
      __syncthreads();
      Prog::forward(t, sc, base);
      if (LAST && GRAD && a.output == TDQ_OUT_EXPVAL && a.n_groups == 1) {
        // one output group: its diagonal weight d(x) gives both the value
        // (sum |psi|^2 d) and lambda = w d psi in one pass over the tile
        const float w = a.gw ? (float)a.gw[b] : 1.f;
        float acc = 0.f;
        for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) {
          const float d = obs_weight(a, 0, gidx(s, base, j, t.L));
          const c2 v = sc.psi[swz(j)];
          acc += (v.x * v.x + v.y * v.y) * d;
          sc.lam[swz(j)] = {w * d * v.x, w * d * v.y};
        }
        acc = warp_sum_f(acc);
        if ((threadIdx.x & 31) == 0) atomicAdd(&s.vsum[0], (double)acc);
        __syncthreads();
        Prog::reverse(t, sc, base);
        for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) {
          const uint32_t x = gidx(s, base, j, t.L);
          gpsi[x] = sc.psi[swz(j)];
          glam[x] = sc.lam[swz(j)];
        }
      } else if (LAST && a.output == TDQ_OUT_EXPVAL) {
        for (int g = 0; g < a.n_groups; g++) {
          float acc = 0.f;
          for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) {
            const c2 v = sc.psi[swz(j)];
            acc += (v.x * v.x + v.y * v.y) * obs_weight(a, g, gidx(s, base, j, t.L));
          }
          acc = warp_sum_f(acc);
          if ((threadIdx.x & 31) == 0) atomicAdd(&s.vsum[g], (double)acc);
        }
        if (GRAD) {
          for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) {
            const uint32_t x = gidx(s, base, j, t.L);
            float d = 0.f;
            for (int g = 0; g < a.n_groups; g++) {
              const float w = a.gw ? (float)a.gw[b * a.n_groups + g] : 1.f;
              d += w * obs_weight(a, g, x);
            }
            const c2 v = sc.psi[swz(j)];
            sc.lam[swz(j)] = {d * v.x, d * v.y};
          }
          __syncthreads();
          Prog::reverse(t, sc, base);
          for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) {
            const uint32_t x = gidx(s, base, j, t.L);
            gpsi[x] = sc.psi[swz(j)];
            glam[x] = sc.lam[swz(j)];
          }
        }
      }
      if (!(LAST && GRAD) && store) {
        for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) gpsi[gidx(s, base, j, t.L)] = sc.psi[swz(j)];
      }
      __syncthreads();
    }
    if (LAST && a.output == TDQ_OUT_EXPVAL) {
      __syncthreads();
      for (int g = threadIdx.x; g < a.n_groups; g += blockDim.x)
        atomicAdd(&t.vals[(int64_t)lr * a.n_groups + g], s.vsum[g]);
    }
    if (GRAD && LAST) Prog::flush(a, t, s, lr);
  });
}

// Reverse pass over the tiles of one pass (passes before the last); psi and
// lambda of the next tile are read while the current one is computed.
template <class Prog>
__device__ __forceinline__ void k1_reverse_body(const SweepArgs& a, const TiledDev& t) {
  extern __shared__ __align__(16) unsigned char raw[];
  const int nb = t.dbl ? 2 : 1;
  const TileShared s = carve(raw, t.k, t.L, nb, nb, t.nrec, t.ndops, a.n_groups, t.gbytes);
  const uint32_t nloc = 1u << t.k;
  const uint32_t dim = 1u << t.n;
  const uint32_t other = (dim - 1u) & ~t.smask;
  k1_for_segments(t, [&](int lr, int tile0, int tile1) {
    const int row = t.row0 + lr;
    const int64_t b = row / a.ps_copies;
    int bad = 0;
    k1_setup(a, t, s, b, 0, &bad);
    c2* gpsi = t.psi + (size_t)lr * dim;
    c2* glam = t.lam + (size_t)lr * dim;
    if (t.dbl && tile0 < tile1) {
      const uint32_t base0 = deposit((uint32_t)tile0, other);
      k1_issue(s.psi, gpsi, s, base0, t.k, t.L);
      k1_issue(s.lam, glam, s, base0, t.k, t.L);
      cp_async_commit();
    }
    for (int tile = tile0, it = 0; tile < tile1; tile++, it++) {
      const uint32_t base = deposit((uint32_t)tile, other);
      TileShared sc = s;
      if (t.dbl) {
        sc.psi = (it & 1) ? s.psi2 : s.psi;
        sc.lam = (it & 1) ? s.lam2 : s.lam;
        if (tile + 1 < tile1) {
          const uint32_t nxt = deposit((uint32_t)(tile + 1), other);
          k1_issue((it & 1) ? s.psi : s.psi2, gpsi, s, nxt, t.k, t.L);
          k1_issue((it & 1) ? s.lam : s.lam2, glam, s, nxt, t.k, t.L);
          cp_async_commit();
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
      } else {  // one buffer per state: load, then compute
        k1_issue(s.psi, gpsi, s, base, t.k, t.L);
        k1_issue(s.lam, glam, s, base, t.k, t.L);
        cp_async_commit();
        cp_async_wait<0>();
      }
      __syncthreads();
      Prog::reverse(t, sc, base);
      for (uint32_t j = threadIdx.x; j < nloc; j += blockDim.x) {
        const uint32_t x = gidx(s, base, j, t.L);
        gpsi[x] = sc.psi[swz(j)];
        glam[x] = sc.lam[swz(j)];
      }
      __syncthreads();
    }
    Prog::flush(a, t, s, lr);
  });
}

}  // namespace tdq
