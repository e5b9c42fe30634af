// Specialised sweep programs (see sweep_jit.h) and their run-time compilation.
#include "sweep_jit.h"

#include <cuda_runtime.h>
#include <nvJitLink.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <map>
#include <mutex>
#include <sstream>
#include <thread>

namespace tdq {

// The device headers the generated source includes, embedded at build time
// (kJitHeaderNames / kJitHeaderSrc / kJitHeaderCount).
#include "jit_headers.inc"

namespace {

// Index bits of one register pass: the group base inserts zeros at the
// pass's tile bits; member j of a group sits at base ^ off(j) (disjoint bits).
struct PassBits {
  int m;
  int lb[4];
  uint32_t off(int j) const {
    uint32_t o = 0;
    for (int i = 0; i < m; i++)
      if ((j >> i) & 1) o |= 1u << lb[i];
    return o;
  }
};

uint32_t swz_host(uint32_t x) { return x ^ ((x >> 4) & 15u); }

PassBits pass_bits(const RegPass& rp) {
  PassBits b{};
  b.m = rp.m;
  for (int i = 0; i < 4; i++) b.lb[i] = rp.lb[i];
  return b;
}

// "gb" computed from the group index, then the swizzled base "sb".
void emit_group_base(std::ostringstream& s, const PassBits& pb) {
  s << "    uint32_t gb = (uint32_t)grp;\n";
  for (int i = 0; i < pb.m; i++) s << "    gb = insert0(gb, " << pb.lb[i] << ");\n";
  s << "    const uint32_t sb = swz(gb);\n";
}

// Loads (store = false) or stores the group's amplitudes; swz is linear over
// XOR and the offsets share no bit with gb, so swz(gb | off) = sb ^ swz(off).
void emit_move(std::ostringstream& s, const PassBits& pb, const char* arr, const char* reg, bool store) {
  for (int j = 0; j < (1 << pb.m); j++) {
    const uint32_t so = swz_host(pb.off(j));
    if (store)
      s << "    " << arr << "[sb ^ " << so << "u] = " << reg << "[" << j << "];\n";
    else
      s << "    " << reg << "[" << j << "] = " << arr << "[sb ^ " << so << "u];\n";
  }
}

// Value of a bit that is not a register bit: a tile bit of the group base
// (l >= 0), else global position p of the tile's base index.
std::string fixed_bit(int l, int p) {
  std::ostringstream s;
  if (l >= 0) s << "((gb >> " << l << ") & 1u)";
  else s << "((base >> " << p << ") & 1u)";
  return s.str();
}

bool dense_kind(int k) {
  return k == K_FUSED || k == K_RX || k == K_RY || k == K_U3 || k == K_H || k == K_X || k == K_Y;
}

// Forward absorption of one decoded op into the register array `a` (M
// register bits).
void emit_fwd_op(std::ostringstream& s, const DOp& d, int M, const char* a) {
  const int k = d.kind;
  s << "    {  // kind " << k << "\n";
  if (dense_kind(k)) {
    s << "      reg_pair<" << M << ", " << (int)d.r0 << ">(" << a << ", mats[" << d.mat << "].m);\n";
  } else if (k == K_CNOT) {  // control p0, target p1 (a register bit)
    if (d.r0 >= 0)
      s << "      swap_ctrl<" << M << ", " << (int)d.r1 << ", " << (int)d.r0 << ">(" << a << ");\n";
    else
      s << "      if (" << fixed_bit(d.l0, d.p0) << ") swap_ctrl<" << M << ", " << (int)d.r1 << ", -1>(" << a << ");\n";
  } else if (k == K_CZ) {
    if (d.r0 >= 0 && d.r1 >= 0)
      s << "      neg_and<" << M << ", " << (int)d.r0 << ", " << (int)d.r1 << ">(" << a << ");\n";
    else if (d.r0 >= 0 || d.r1 >= 0) {
      const int r = d.r0 >= 0 ? d.r0 : d.r1, l = d.r0 >= 0 ? d.l1 : d.l0, pp = d.r0 >= 0 ? d.p1 : d.p0;
      s << "      if (" << fixed_bit(l, pp) << ") neg_and<" << M << ", " << r << ", " << r << ">(" << a << ");\n";
    } else {
      s << "      if (" << fixed_bit(d.l0, d.p0) << " & " << fixed_bit(d.l1, d.p1) << ")\n"
        << "        for (int j = 0; j < " << (1 << M) << "; j++) " << a << "[j] = {-" << a << "[j].x, -" << a
        << "[j].y};\n";
    }
  } else {  // diagonal phases: RZ / Z (one bit), RZZ (parity of two bits)
    const bool two = k == K_RZZ;
    s << "      c2 d0 = mats[" << d.mat << "].m.m00, d1 = mats[" << d.mat << "].m.m11;\n";
    std::string fx;
    if (d.r0 < 0) fx = fixed_bit(d.l0, d.p0);
    if (two && d.r1 < 0) fx = fx.empty() ? fixed_bit(d.l1, d.p1) : "(" + fx + " ^ " + fixed_bit(d.l1, d.p1) + ")";
    if (!fx.empty()) s << "      if (" << fx << ") { const c2 t = d0; d0 = d1; d1 = t; }\n";
    s << "      diag_par<" << M << ", " << (int)d.r0 << ", " << (two ? (int)d.r1 : -1) << ">(" << a
      << ", d0, d1);\n";
  }
  s << "    }\n";
}

// Reverse step of one op on p[], l[]: gradient shares into gs<i> variables.
void emit_rev_op(std::ostringstream& s, const DOp& d, int M, const std::vector<int>& gvar) {
  const int k = d.kind;
  s << "    {  // kind " << k << "\n";
  auto add = [&](int j, const char* expr) {
    if (j < d.nang && d.slot[j] >= 0 && gvar[j] >= 0)
      s << "      gs" << gvar[j] / 32 << "[" << gvar[j] % 32 << "] += " << expr << ";\n";
  };
  if (k == K_CNOT || k == K_CZ) {  // self-inverse: the forward action on both states
    s << "    }\n";
    emit_fwd_op(s, d, M, "p");
    emit_fwd_op(s, d, M, "l");
    return;
  } else if (!dense_kind(k)) {  // RZ / Z / RZZ
    const bool two = k == K_RZZ;
    s << "      c2 d0 = mats[" << d.mat << "].m.m00, d1 = mats[" << d.mat << "].m.m11;\n"
      << "      d0.y = -d0.y; d1.y = -d1.y;\n";
    std::string fx;
    if (d.r0 < 0) fx = fixed_bit(d.l0, d.p0);
    if (two && d.r1 < 0) fx = fx.empty() ? fixed_bit(d.l1, d.p1) : "(" + fx + " ^ " + fixed_bit(d.l1, d.p1) + ")";
    if (!fx.empty()) s << "      const bool fx = " << fx << ";\n      if (fx) { const c2 t = d0; d0 = d1; d1 = t; }\n";
    s << "      float acc = 0.f;\n"
      << "      diag_par_adj<" << M << ", " << (int)d.r0 << ", " << (two ? (int)d.r1 : -1)
      << ">(p, l, d0, d1, acc);\n";
    add(0, fx.empty() ? "acc" : "(fx ? -acc : acc)");
  } else {
    s << "      float g[3] = {0.f, 0.f, 0.f};\n"
      << "      reg_adj_1q<" << M << ", " << (int)d.r0 << ">(p, l, " << k << ", mats[" << d.mat << "], g);\n";
    add(0, "g[0]");
    add(1, "g[1]");
    add(2, "g[2]");
  }
  s << "    }\n";
}

// One forward register pass as a group loop over the tile (or state) in
// `st` of 2^k amplitudes; ops [op0 + rp.op_begin, op0 + rp.op_end) of dops.
void emit_fwd_pass(std::ostringstream& s, const RegPass& rp, const std::vector<DOp>& dops, int op0, int k,
                   const char* st) {
  const PassBits pb = pass_bits(rp);
  s << "  for (int grp = threadIdx.x; grp < " << (1 << (k - pb.m)) << "; grp += blockDim.x) {\n";
  emit_group_base(s, pb);
  s << "    c2 a[" << (1 << pb.m) << "];\n";
  emit_move(s, pb, st, "a", false);
  for (int o = rp.op_begin; o < rp.op_end; o++) emit_fwd_op(s, dops[op0 + o], pb.m, "a");
  emit_move(s, pb, st, "a", true);
  s << "  }\n  __syncthreads();\n";
}

// One reverse register pass: gradient shares go to accumulator index
// acc_index(op, angle) of the per-warp rows gpart[warp * stride + index],
// reduced over the warp for up to 32 accumulators at once (grad_share_multi;
// their index tables are declared into `decl`).
template <class F>
void emit_rev_pass(std::ostringstream& s, std::ostringstream& decl, int* uid, const RegPass& rp,
                   const std::vector<DOp>& dops, int op0, int k, const char* sp, const char* sl, int stride,
                   F acc_index) {
  const PassBits pb = pass_bits(rp);
  // The pass's gradient shares, summed per accumulator index in registers
  // gs<chunk>[position] (a chunk holds at most 32 distinct indices; shares of
  // gates that use one parameter add into one register), then reduced over
  // the warp a chunk at a time by grad_share_multi, whose K lanes add to
  // gpart[warp * stride + table[j]] in one instruction (a read-add-write of
  // shared memory): no table may hold an index twice, or two lanes would read
  // the same old value and one addition would be lost.  A chunk of g indices
  // is padded to K = 2^ceil(log2 g) with indices the chunk does not use (the
  // padding lanes add zero there); if fewer than K - g are free, it is cut
  // into power-of-two chunks instead.  gv holds 32 * chunk + position.
  std::vector<std::vector<int>> gv(rp.op_end - rp.op_begin, std::vector<int>(3, -1));
  std::vector<std::vector<int>> chunks;  // accumulator indices, by position
  std::vector<int> open_idx;             // distinct indices of the chunk being filled
  std::vector<std::pair<std::pair<int, int>, int>> open_sh;  // ((op, angle), position in open_idx)
  auto close_chunk = [&] {
    int g = (int)open_idx.size();
    int at = 0;
    while (g > 0) {
      int kk = 1;
      while (kk < g) kk <<= 1;
      if (kk - g > stride - g) kk >>= 1;  // too few free indices: the largest power of two below g
      const int take = std::min(kk, g);
      const int c = (int)chunks.size();
      chunks.emplace_back(open_idx.begin() + at, open_idx.begin() + at + take);
      for (const auto& sh : open_sh)
        if (sh.second >= at && sh.second < at + take) gv[sh.first.first][sh.first.second] = 32 * c + sh.second - at;
      at += take;
      g -= take;
    }
    open_idx.clear();
    open_sh.clear();
  };
  for (int o = rp.op_begin; o < rp.op_end; o++) {
    const DOp& d = dops[op0 + o];
    for (int j = 0; j < d.nang && j < 3; j++)
      if (d.slot[j] >= 0) {
        const int idx = acc_index(op0 + o, j);
        auto it = std::find(open_idx.begin(), open_idx.end(), idx);
        if (it == open_idx.end() && open_idx.size() == 32) {
          close_chunk();
          it = open_idx.end();
        }
        if (it == open_idx.end()) {
          open_idx.push_back(idx);
          it = open_idx.end() - 1;
        }
        open_sh.push_back({{o - rp.op_begin, j}, (int)(it - open_idx.begin())});
      }
  }
  close_chunk();
  std::vector<int> chunk_k;  // padded size of each chunk
  for (auto& ch : chunks) {
    int kk = 1;
    while (kk < (int)ch.size()) kk <<= 1;
    chunk_k.push_back(kk);
    // padding: the lowest accumulator indices the chunk does not use
    for (int cand = 0; (int)ch.size() < kk && cand < stride; cand++)
      if (std::find(ch.begin(), ch.end(), cand) == ch.end()) ch.push_back(cand);
  }
  s << "  {\n";
  for (size_t c = 0; c < chunk_k.size(); c++) {
    s << "  float gs" << c << "[" << chunk_k[c] << "] = {";
    for (int j = 0; j < chunk_k[c]; j++) s << (j ? ", " : "") << "0.f";
    s << "};\n";
  }
  s << "  for (int grp = threadIdx.x; grp < " << (1 << (k - pb.m)) << "; grp += blockDim.x) {\n";
  emit_group_base(s, pb);
  s << "    c2 p[" << (1 << pb.m) << "], l[" << (1 << pb.m) << "];\n";
  emit_move(s, pb, sp, "p", false);
  emit_move(s, pb, sl, "l", false);
  for (int o = rp.op_end - 1; o >= rp.op_begin; o--) emit_rev_op(s, dops[op0 + o], pb.m, gv[o - rp.op_begin]);
  emit_move(s, pb, sp, "p", true);
  emit_move(s, pb, sl, "l", true);
  s << "  }\n";
  for (size_t c = 0; c < chunk_k.size(); c++) {
    const int id = (*uid)++;
    decl << "__constant__ int tdq_gi_" << id << "[" << chunk_k[c] << "] = {";
    for (int j = 0; j < chunk_k[c]; j++) decl << (j ? ", " : "") << chunks[c][j];
    decl << "};\n";
    s << "  grad_share_multi<" << chunk_k[c] << ">(gpart, " << stride << ", tdq_gi_" << id << ", gs" << c << ");\n";
  }
  s << "  __syncthreads();\n  }\n";
}

}  // namespace

// The program struct `sname` of one circuit (forward passes [0, npf), reverse
// passes [npf, npf + npb)); constant tables go to decl, numbered from *uid.
static void k2_prog_struct(std::ostringstream& s, std::ostringstream& decl, int* uid, const Program& prog, int npf,
                           int npb, int P, int n, const std::string& sname) {
  s << "struct " << sname << " {\n"
    << "  static constexpr bool kSpecialised = true;\n  const DOp* dops;\n";
  s << "  template <int MF>\n  __device__ __forceinline__ void forward(c2* psi, const OpMat* mats, int) const {\n"
    << "  const uint32_t base = 0u;\n";
  for (int pi = 0; pi < npf; pi++) {
    s << "  // forward pass " << pi << "\n";
    emit_fwd_pass(s, prog.passes[pi], prog.dops, 0, n, "psi");
  }
  s << "  }\n";
  s << "  template <int MB>\n  __device__ __forceinline__ void reverse(c2* psi, c2* lam, const OpMat* mats, int, "
       "double*, float* gpart) const {\n  const uint32_t base = 0u;\n";
  for (int pi = npf + npb - 1; pi >= npf; pi--) {
    s << "  // reverse pass " << pi << "\n";
    emit_rev_pass(s, decl, uid, prog.passes[pi], prog.dops, 0, n, "psi", "lam", P,
                  [&](int o, int j) { return (int)prog.dops[o].slot[j]; });
  }
  s << "  }\n};\n";
}

std::string k2_specialised_source(const Program& prog, int npf, int npb, int mf, int mb, int nthreads,
                                  int P, int n, const char* name) {
  std::ostringstream s, decl;
  int uid = 0;
  k2_prog_struct(s, decl, &uid, prog, npf, npb, P, n, "SpecProg");
  s << "}  // namespace tdq\n";
  std::ostringstream out;
  out << "#include \"k2_body.cuh\"\nnamespace tdq {\n" << decl.str() << s.str();
  const int minb = nthreads >= 256 ? 2 : 1;
  out << "extern \"C\" __global__ void __launch_bounds__(" << nthreads << ", " << minb << ") " << name
    << "(tdq::SweepArgs a, const tdq::DOp* gdops, int ndops, const int* rec_ptr, const int* rec_ops, int nrec) {\n"
    << "  tdq::k2_body<" << mf << ", " << mb << ", " << (npb > 0 ? "true" : "false")
    << ", tdq::SpecProg>(a, tdq::SpecProg{nullptr}, gdops, 0, rec_ptr, rec_ops, nrec, blockIdx.x);\n}\n";
  return out.str();
}

std::vector<std::string> k2_multi_modules(const std::vector<K2Part>& parts, bool grad, int nthreads,
                                          const char* name) {
  std::vector<std::string> mods(1);
  int uid = 0;  // constant tables numbered across modules: their names stay unique at link time
  for (size_t c = 0; c < parts.size(); c++) {
    std::ostringstream s, decl;
    k2_prog_struct(s, decl, &uid, *parts[c].prog, parts[c].npf, parts[c].npb, parts[c].P, parts[c].n,
                   "SpecProg_" + std::to_string(c));
    std::ostringstream out;
    out << "#include \"k2_body.cuh\"\nnamespace tdq {\n" << decl.str() << s.str() << "}  // namespace tdq\n";
    // the circuit's row body: a function of its own, linked to the launch module
    out << "__device__ __noinline__ void tdq_multi_row_" << c
        << "(const tdq::SweepArgs& a, const tdq::MultiCirc& m, int r) {\n  tdq::k2_body<" << parts[c].mf << ", "
        << parts[c].mb << ", " << (grad ? "true" : "false") << ", tdq::SpecProg_" << c << ">(a, tdq::SpecProg_"
        << c << "{nullptr}, nullptr, 0, m.rec_ptr, m.rec_ops, m.nrec, r);\n}\n";
    mods.push_back(out.str());
  }
  std::ostringstream out;
  out << "#include \"sweep_common.cuh\"\n";
  for (size_t c = 0; c < parts.size(); c++)
    out << "__device__ void tdq_multi_row_" << c << "(const tdq::SweepArgs& a, const tdq::MultiCirc& m, int r);\n";
  // persistent CTAs take (circuit, row) items from a counter until none is left
  out << "extern \"C\" __global__ void __launch_bounds__(" << nthreads << ", 1) " << name
      << "(const tdq::MultiCirc* __restrict__ mc, const int2* __restrict__ items, int n_items, int* next,\n"
      << "    const float* params, const float* inputs, double* values, const double* gw, float* grads) {\n"
      << "  __shared__ int s_item;\n"
      << "  for (;;) {\n"
      << "    __syncthreads();\n"
      << "    if (threadIdx.x == 0) s_item = atomicAdd(next, 1);\n"
      << "    __syncthreads();\n"
      << "    const int it = s_item;\n"
      << "    if (it >= n_items) return;\n"
      << "    const int2 w = items[it];\n"
      << "    const tdq::MultiCirc& m = mc[w.x];\n"
      << "    tdq::SweepArgs a = m.a;\n"
      << "    a.params = params + m.p_off;\n"
      << "    a.inputs = inputs ? inputs + m.x_off : nullptr;\n"
      << "    a.values = values + m.v_off;\n"
      << "    a.gw = gw ? gw + m.v_off : nullptr;\n"
      << "    a.grads = grads ? grads + m.g_off : nullptr;\n"
      << "    switch (w.x) {\n";
  for (size_t c = 0; c < parts.size(); c++)
    out << "      case " << c << ": tdq_multi_row_" << c << "(a, m, w.y); break;\n";
  out << "      default: break;\n    }\n  }\n}\n";
  mods[0] = out.str();
  return mods;
}

std::string k1_specialised_source(const TiledSweep& t, const Program& prog, int nthreads, int nthreads_r,
                                  std::vector<int>* nacc) {
  std::ostringstream s, decl;
  int uid = 0;
  const int np = (int)t.passes.size();
  nacc->assign(np, 0);
  for (int p = 0; p < np; p++) {
    const int d0 = t.dop_begin[p];
    // gradient accumulators of the pass: one per (reverse op, angle) with a slot
    std::map<std::pair<int, int>, int> acc;
    std::vector<int> slots;
    if (t.adj)
      for (int q = t.bp_begin[p]; q < t.bp_end[p]; q++)
        for (int o = prog.passes[q].op_begin; o < prog.passes[q].op_end; o++) {
          const DOp& d = prog.dops[d0 + o];
          for (int j = 0; j < d.nang && j < 3; j++)
            if (d.slot[j] >= 0) {
              acc[{d0 + o, j}] = (int)slots.size();
              slots.push_back(d.slot[j]);
            }
        }
    (*nacc)[p] = (int)slots.size();
    const int na = std::max(1, (int)slots.size());
    s << "__constant__ int tdq_slots_" << p << "[" << na << "] = {";
    for (int i = 0; i < na; i++) s << (i ? ", " : "") << (i < (int)slots.size() ? slots[i] : 0);
    s << "};\n";
    s << "struct TilePass" << p << " {\n";
    s << "  __device__ __forceinline__ static void forward(const TiledDev&, const TileShared& s, uint32_t base) {\n"
      << "  c2* psi = s.psi;\n  const OpMat* mats = s.mats;\n";
    for (int q = t.fp_begin[p]; q < t.fp_end[p]; q++) emit_fwd_pass(s, prog.passes[q], prog.dops, d0, t.k, "psi");
    s << "  }\n";
    s << "  __device__ __forceinline__ static void reverse(const TiledDev&, const TileShared& s, uint32_t base) {\n"
      << "  c2* psi = s.psi;\n  c2* lam = s.lam;\n  const OpMat* mats = s.mats;\n"
      << "  float* gpart = reinterpret_cast<float*>(s.gpart);\n";
    for (int q = t.bp_end[p] - 1; q >= t.bp_begin[p]; q--)
      emit_rev_pass(s, decl, &uid, prog.passes[q], prog.dops, d0, t.k, "psi", "lam", na,
                    [&](int o, int j) { return acc.at({o, j}); });
    s << "  }\n";
    s << "  __device__ __forceinline__ static void flush(const SweepArgs& a, const TiledDev& t, const TileShared& s, "
         "int lr) {\n"
      << "  __syncthreads();\n  const float* gp = reinterpret_cast<const float*>(s.gpart);\n"
      << "  const int nw = blockDim.x >> 5;\n"
      << "  for (int i = threadIdx.x; i < " << (int)slots.size() << "; i += blockDim.x) {\n"
      << "    double v = 0.0;\n    for (int w = 0; w < nw; w++) v += (double)gp[w * " << na << " + i];\n"
      << "    atomicAdd(&t.gacc[(int64_t)lr * a.P + tdq_slots_" << p << "[i]], v);\n  }\n  }\n};\n";
  }
  s << "}  // namespace tdq\n";
  std::ostringstream out;
  out << "#include \"k1_body.cuh\"\nnamespace tdq {\n" << decl.str() << s.str();
  const int minb = nthreads >= 256 ? 2 : 1;
  for (int p = 0; p < np; p++) {
    const bool f = p == 0, l = p == np - 1;
    out << "extern \"C\" __global__ void __launch_bounds__(" << nthreads << ", " << minb << ") tdq_k1f_" << p
      << "(tdq::SweepArgs a, tdq::TiledDev t, int store) {\n  tdq::k1_forward_body<" << (f ? "true" : "false") << ", "
      << (l ? "true" : "false") << ", " << ((l && t.adj) ? "true" : "false") << ", tdq::TilePass" << p
      << ">(a, t, store);\n}\n";
    if (t.adj && !l)
      out << "extern \"C\" __global__ void __launch_bounds__(" << nthreads_r << ", " << (nthreads_r <= 256 ? 2 : 1)
          << ") tdq_k1r_" << p
        << "(tdq::SweepArgs a, tdq::TiledDev t) {\n  tdq::k1_reverse_body<tdq::TilePass" << p << ">(a, t);\n}\n";
  }
  return out.str();
}

namespace {

struct JitCache {
  std::mutex mu;
  std::map<std::string, cudaLibrary_t> libs;  // by source
};

JitCache& cache() {
  static JitCache* c = new JitCache();  // never destroyed: kernels outlive static teardown order
  return *c;
}

std::string nvrtc_log(nvrtcProgram p) {
  size_t n = 0;
  if (nvrtcGetProgramLogSize(p, &n) != NVRTC_SUCCESS || n == 0) return "";
  std::string log(n, '\0');
  nvrtcGetProgramLog(p, &log[0]);
  return log;
}

}  // namespace

tdq_status jit_kernel(const std::string& src, const char* name, const void** kernel) {
  *kernel = nullptr;
  int dev = 0;
  TDQ_CUDA_TRY(cudaGetDevice(&dev));
  int maj = 0, min = 0;
  TDQ_CUDA_TRY(cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev));
  TDQ_CUDA_TRY(cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev));
  if (maj != 10 || min != 3)
    return fail(TDQ_ERR_UNSUPPORTED, "specialised sweep: built for sm_103a, device is sm_" +
                                         std::to_string(maj) + std::to_string(min));
  // one compilation per source, all its kernels; NVRTC runs outside the lock
  // so that different sources compile concurrently
  JitCache& C = cache();
  cudaLibrary_t lib = nullptr;
  {
    std::lock_guard<std::mutex> lk(C.mu);
    auto it = C.libs.find(src);
    if (it != C.libs.end()) lib = it->second;
  }
  if (!lib) {
    nvrtcProgram p;
    if (nvrtcCreateProgram(&p, src.c_str(), "tdq_specialised.cu", kJitHeaderCount, kJitHeaderSrc,
                           kJitHeaderNames) != NVRTC_SUCCESS)
      return fail(TDQ_ERR_CUDA, "specialised sweep: nvrtcCreateProgram failed");
    const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "-lineinfo"};
    const nvrtcResult r = nvrtcCompileProgram(p, 4, opts);
    const std::string log = nvrtc_log(p);
    if (std::getenv("TDQ_JIT_LOG") && !log.empty()) fprintf(stderr, "%s\n", log.c_str());
    if (r != NVRTC_SUCCESS) {
      nvrtcDestroyProgram(&p);
      return fail(TDQ_ERR_CUDA, std::string("specialised sweep: compilation failed: ") + nvrtcGetErrorString(r) +
                                    "\n" + log.substr(0, 4000));
    }
    size_t n = 0;
    nvrtcGetCUBINSize(p, &n);
    std::string cubin(n, '\0');
    nvrtcGetCUBIN(p, &cubin[0]);
    nvrtcDestroyProgram(&p);
    TDQ_CUDA_TRY(cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
    std::lock_guard<std::mutex> lk(C.mu);
    auto ins = C.libs.emplace(src, lib);
    if (!ins.second) {  // another thread compiled the same source meanwhile
      cudaLibraryUnload(lib);
      lib = ins.first->second;
    }
  }
  cudaKernel_t k = nullptr;
  TDQ_CUDA_TRY(cudaLibraryGetKernel(&k, lib, name));
  *kernel = reinterpret_cast<const void*>(k);
  return TDQ_OK;
}


// One module compiled to relocatable device code (a cubin for linking), its
// functions held to maxrreg registers (0: no limit).
static tdq_status jit_module(const std::string& src, int maxrreg, std::string* cubin, std::string* err) {
  nvrtcProgram p;
  if (nvrtcCreateProgram(&p, src.c_str(), "tdq_module.cu", kJitHeaderCount, kJitHeaderSrc, kJitHeaderNames) !=
      NVRTC_SUCCESS) {
    *err = "nvrtcCreateProgram failed";
    return TDQ_ERR_CUDA;
  }
  const std::string rr = "--maxrregcount=" + std::to_string(maxrreg);
  const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-default-device", "-lineinfo", "-rdc=true", rr.c_str()};
  const nvrtcResult r = nvrtcCompileProgram(p, maxrreg > 0 ? 6 : 5, opts);
  if (r != NVRTC_SUCCESS) {
    *err = std::string("compilation failed: ") + nvrtcGetErrorString(r) + "\n" + nvrtc_log(p).substr(0, 4000);
    nvrtcDestroyProgram(&p);
    return TDQ_ERR_CUDA;
  }
  size_t n = 0;
  nvrtcGetCUBINSize(p, &n);
  cubin->assign(n, '\0');
  nvrtcGetCUBIN(p, &(*cubin)[0]);
  nvrtcDestroyProgram(&p);
  return TDQ_OK;
}

tdq_status jit_link_kernel(const std::vector<std::string>& mods, const char* name, int maxrreg, const void** kernel) {
  *kernel = nullptr;
  int dev = 0;
  TDQ_CUDA_TRY(cudaGetDevice(&dev));
  int maj = 0, min = 0;
  TDQ_CUDA_TRY(cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev));
  TDQ_CUDA_TRY(cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev));
  if (maj != 10 || min != 3)
    return fail(TDQ_ERR_UNSUPPORTED, "specialised sweep: built for sm_103a, device is sm_" + std::to_string(maj) +
                                         std::to_string(min));
  std::string key = std::to_string(maxrreg) + '\0';
  for (const std::string& m : mods) {
    key += m;
    key.push_back('\0');
  }
  JitCache& C = cache();
  cudaLibrary_t lib = nullptr;
  {
    std::lock_guard<std::mutex> lk(C.mu);
    auto it = C.libs.find(key);
    if (it != C.libs.end()) lib = it->second;
  }
  if (!lib) {
    // every module on its own host thread, then one link
    std::vector<std::string> cubins(mods.size()), errs(mods.size());
    std::vector<tdq_status> st(mods.size(), TDQ_OK);
    std::atomic<size_t> next{0};
    const size_t nt = std::max<size_t>(1, std::min<size_t>(mods.size(), std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (size_t w = 0; w < nt; w++)
      pool.emplace_back([&] {
        for (size_t i = next++; i < mods.size(); i = next++) {
          try {
            st[i] = jit_module(mods[i], maxrreg, &cubins[i], &errs[i]);
          } catch (...) {
            st[i] = TDQ_ERR_OOM;
            errs[i] = "host allocation";
          }
        }
      });
    for (auto& t : pool) t.join();
    for (size_t i = 0; i < mods.size(); i++)
      if (st[i] != TDQ_OK) return fail(st[i], "specialised sweep, module " + std::to_string(i) + ": " + errs[i]);
    nvJitLinkHandle h;
    const char* lopts[] = {"-arch=sm_103a"};
    if (nvJitLinkCreate(&h, 1, lopts) != NVJITLINK_SUCCESS) return fail(TDQ_ERR_CUDA, "nvJitLinkCreate failed");
    auto link_fail = [&](const std::string& what) {
      size_t n = 0;
      std::string log;
      if (nvJitLinkGetErrorLogSize(h, &n) == NVJITLINK_SUCCESS && n > 1) {
        log.assign(n, '\0');
        nvJitLinkGetErrorLog(h, &log[0]);
      }
      nvJitLinkDestroy(&h);
      return fail(TDQ_ERR_CUDA, "specialised sweep: " + what + "\n" + log.substr(0, 4000));
    };
    for (size_t i = 0; i < cubins.size(); i++)
      if (nvJitLinkAddData(h, NVJITLINK_INPUT_CUBIN, cubins[i].data(), cubins[i].size(),
                           ("module" + std::to_string(i)).c_str()) != NVJITLINK_SUCCESS)
        return link_fail("adding module " + std::to_string(i));
    if (nvJitLinkComplete(h) != NVJITLINK_SUCCESS) return link_fail("link failed");
    size_t n = 0;
    if (nvJitLinkGetLinkedCubinSize(h, &n) != NVJITLINK_SUCCESS) return link_fail("linked size");
    std::string cubin(n, '\0');
    if (nvJitLinkGetLinkedCubin(h, &cubin[0]) != NVJITLINK_SUCCESS) return link_fail("linked cubin");
    nvJitLinkDestroy(&h);
    TDQ_CUDA_TRY(cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
    std::lock_guard<std::mutex> lk(C.mu);
    auto ins = C.libs.emplace(key, lib);
    if (!ins.second) {
      cudaLibraryUnload(lib);
      lib = ins.first->second;
    }
  }
  cudaKernel_t k = nullptr;
  TDQ_CUDA_TRY(cudaLibraryGetKernel(&k, lib, name));
  *kernel = reinterpret_cast<const void*>(k);
  return TDQ_OK;
}

}  // namespace tdq
