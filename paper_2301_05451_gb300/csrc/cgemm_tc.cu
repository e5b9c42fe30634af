// K3: 3xTF32 complex NT product on tcgen05 tensor cores (see cgemm_tc.cuh).
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched at run time)
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "cgemm_tc.cuh"
#include "tdq_internal.h"

namespace tdq {

namespace {

constexpr int BM = 128, BN = 64, BK = 8;  // tile rows (i), cols (j), complex k per block
constexpr int kConv = 512;              // converter / epilogue threads: warps 0..15
constexpr int kConvWarps = kConv / 32;
// + warp kConvWarps (the tensor-core issuer) and warp kConvWarps + 1 (the TMA producer)
constexpr int kThreads = kConv + 64;
// The converters work in kGroups groups of kGroupWarps warps; group g
// converts the k-blocks kb = g (mod kGroups), one whole k-block at a time, so
// that the groups' k-blocks are in flight together.  Per k-block a group
// thread converts kXP k-pairs of X and kYP of Y.
constexpr int kGroups = 4;
constexpr int kGroupWarps = kConvWarps / kGroups;
constexpr int kGroupThreads = kGroupWarps * 32;
constexpr int kXP = BM * BK / 2 / kGroupThreads, kYP = BN * BK / 2 / kGroupThreads;
static_assert(kXP * kGroupThreads == BM * BK / 2 && kYP * kGroupThreads == BN * BK / 2, "k-pairs per group thread");
static_assert(kGroupWarps == 4, "a group's warps cover the four TMEM lane quarters");
// TMEM read-out: warp w reads lanes 32 (w % 4) .. and a group of kColW columns
constexpr int kColW = BN / (kConvWarps / 4);
constexpr int kXPlane = BM * BK * 4;  // bytes: one real TF32 plane of the X tile
constexpr int kYPlane = BN * BK * 4;
constexpr int kStageBytes = 4 * kXPlane + 4 * kYPlane;  // re_hi, re_lo, im_hi, im_lo of X and Y
constexpr int kStages = 7;  // TF32 plane stages in flight on the tensor cores
// raw operand k-blocks in flight (TMA ring ahead of the split into planes)
constexpr int kRing = 4;
constexpr int kRawX = BM * BK * 8, kRawY = BN * BK * 8;  // bytes of one raw (complex) k-block
constexpr int kRawBytes = kRing * (kRawX + kRawY);
// Shared memory per CTA: the plane stages and the raw ring (the FP32 sums
// live in TMEM).  It is above half the SM's shared memory, so one CTA runs
// per SM -- it then owns all 512 TMEM columns and tcgen05.alloc never waits
// for another CTA.
constexpr int kSmemBytes = kStages * kStageBytes + kRawBytes;
static_assert(kSmemBytes <= 227 * 1024, "K3 shared memory");
static_assert(kSmemBytes > 114 * 1024, "K3: one CTA per SM");
constexpr uint32_t kTmemCols = 512;
// six accumulators of 64 columns: hi*hi terms of Re+, Re-, Im, then the
// hi*lo + lo*hi correction terms of the same three
constexpr uint32_t kAccStride = 64;
constexpr int kChunk = 16;  // k-blocks accumulated in TMEM before a flush to the FP32 sums
// the FP32 sums of the flushed chunks in the last 128 TMEM columns: Re of the
// tile's 64 columns, then Im
constexpr uint32_t kSumRe = 6 * kAccStride, kSumIm = kSumRe + BN;
static_assert(kSumIm + BN <= kTmemCols, "FP32 sums in TMEM");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of (row, k) in a K-major operand plane without swizzling:
// core matrices of 8 rows x 16 bytes stored contiguously; the two
// k-adjacent cores 128 bytes apart (leading byte offset), 8-row groups 256
// bytes apart (stride byte offset).
__device__ __forceinline__ uint32_t plane_off(int row, int k) {
  return (uint32_t)((row >> 3) * 256 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and
// stride byte offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((256u >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(void* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Tiled TMA load of a box of a 3-D tensor map (x innermost) into shared
// memory; completion is counted in bytes on mbarrier `bar`.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, void* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(void* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(a), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for the phase of `bar` with the given parity: polls
// mbarrier.try_wait (no suspend-time hint) and gives up after limit_ns of the
// global timer.  The timer is read only once the first poll has failed, so a
// phase that is already complete costs one poll.
__device__ __forceinline__ bool mbar_wait(void* bar, uint32_t parity, uint64_t limit_ns) {
  const uint32_t a = smem_u32(bar);
  if (mbar_try(a, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try(a, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ uint32_t scat(uint32_t x, const int8_t* pos, int n) {
  uint32_t r = 0;
  for (int b = 0; b < n; b++) r |= ((x >> b) & 1u) << pos[b];
  return r;
}

// X, Y: tensor maps over the operands as float [batch][rows][2K] (re, im
// interleaved), boxes of BK complex by BM (X) / BN (Y) rows.
__global__ void __launch_bounds__(kThreads, 1)
    k_cgemm_tc(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmy, float2* out,
               int64_t os, int K, CgemmOut map, int* status, uint64_t wait_ns) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // full[s]: a converter group wrote stage s (one arrival per warp of the group);
  // empty[s]: the tensor cores are done with it (commit); cdone: a chunk's
  // products are in TMEM (commit); flushed: the converters read the chunk out
  // (one arrival per converter warp); fin: every product issued has completed
  // (commit)
  // raw_full[r]: the TMA load of ring slot r landed (byte count); raw_empty[r]:
  // the converters read it (one arrival per converter warp)
  // cdone[c & 1] completes chunk c: the group that flushes chunk c waits for
  // completion c / 2 of its barrier, and chunk c - 2's completion is certain
  // by then (chunk c's first products needed chunk c - 1 flushed), so a
  // parity wait never looks two phases back
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], cdone[2], flushed, fin;
  __shared__ __align__(8) uint64_t raw_full[kRing], raw_empty[kRing];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const int nkb = K / BK;

  if (tid == 0) {
    for (int s = 0; s < kStages; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(kGroupWarps));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&cdone[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&cdone[1])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&flushed)), "r"(kGroupWarps));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fin)));
    for (int r = 0; r < kRing; r++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&raw_full[r])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&raw_empty[r])), "r"(kGroupWarps));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
  }
  if (warp == kConvWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  // raw ring slot r: the TMA boxes of one k-block, X [BM rows][BK complex]
  // then Y [BN rows][BK complex], dense.  Group thread gt converts the
  // k-pairs q = gt + kGroupThreads u -- X: u < kXP, Y: u < kYP; row q >> 2,
  // k 2 (q & 3) -- at plane offsets fixed per thread.
  unsigned char* raw = smem + kStages * kStageBytes;
  const int grp = warp / kGroupWarps, gt = tid - grp * kGroupThreads;
  uint32_t xoff[kXP], yoff[kYP];
#pragma unroll
  for (int u = 0; u < kXP; u++) {
    const int q = gt + kGroupThreads * u, r = q >> 2, k = 2 * (q & 3);
    xoff[u] = plane_off(r, k);
  }
#pragma unroll
  for (int u = 0; u < kYP; u++) {
    const int q = gt + kGroupThreads * u, r = q >> 2, k = 2 * (q & 3);
    yoff[u] = plane_off(r, k);
  }
  // hi / lo TF32 split of two complex values (re0, im0, re1, im1) into the
  // four planes at byte offset o (the two k are adjacent: 8-byte stores)
  auto split2 = [&](unsigned char* pl, int plane_bytes, uint32_t o, float4 v) {
    const float rh0 = tf32_rna(v.x), ih0 = tf32_rna(v.y), rh1 = tf32_rna(v.z), ih1 = tf32_rna(v.w);
    *reinterpret_cast<float2*>(pl + 0 * plane_bytes + o) = make_float2(rh0, rh1);
    *reinterpret_cast<float2*>(pl + 1 * plane_bytes + o) = make_float2(tf32_rna(v.x - rh0), tf32_rna(v.z - rh1));
    *reinterpret_cast<float2*>(pl + 2 * plane_bytes + o) = make_float2(ih0, ih1);
    *reinterpret_cast<float2*>(pl + 3 * plane_bytes + o) = make_float2(tf32_rna(v.y - ih0), tf32_rna(v.w - ih1));
  };
  // raw ring slot of k-block kb -> shared stage: TF32 hi / lo planes of re and im
  auto store = [&](int stage, int kb) {
    unsigned char* base = smem + stage * kStageBytes;
    const float4* rx = reinterpret_cast<const float4*>(raw + (kb % kRing) * (kRawX + kRawY));
    const float4* ry = reinterpret_cast<const float4*>(raw + (kb % kRing) * (kRawX + kRawY) + kRawX);
    float4 vx[kXP], vy[kYP];  // all loads first: one latency for the k-block
#pragma unroll
    for (int u = 0; u < kXP; u++) vx[u] = rx[gt + kGroupThreads * u];
#pragma unroll
    for (int u = 0; u < kYP; u++) vy[u] = ry[gt + kGroupThreads * u];
#pragma unroll
    for (int u = 0; u < kXP; u++) split2(base, kXPlane, xoff[u], vx[u]);
#pragma unroll
    for (int u = 0; u < kYP; u++) split2(base + 4 * kXPlane, kYPlane, yoff[u], vy[u]);
  };

  // FP32 sums of the flushed chunks (TMEM): thread (warp w, lane l) owns row
  // 32 (w % 4) + l (its TMEM lane) and columns [kColW (w / 4), kColW (w / 4 + 1))
  const int row = (warp & 3) * 32 + lane;
  const int col0 = (warp >> 2) * kColW;
  const uint32_t lane_addr = (uint32_t)((warp & 3) * 32) << 16;
  auto ld16 = [&](uint32_t col, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(tmem + lane_addr + col));
  };
  auto st16 = [&](uint32_t col, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            tmem + lane_addr + col),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
  };
  // TMEM accumulators -> registers -> FP32 sums (round to nearest) in TMEM,
  // for this thread's row
  auto flush = [&](bool first, int cb, int ce) {
#pragma unroll 1
    for (int c = cb; c < ce; c += 16) {
      uint32_t a[16], b[16];
      float re[16], im[16];
      ld16(0 * kAccStride + c, a);
      ld16(3 * kAccStride + c, b);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int t = 0; t < 16; t++) re[t] = __uint_as_float(a[t]) + __uint_as_float(b[t]);
      ld16(1 * kAccStride + c, a);
      ld16(4 * kAccStride + c, b);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int t = 0; t < 16; t++) re[t] -= __uint_as_float(a[t]) + __uint_as_float(b[t]);
      ld16(2 * kAccStride + c, a);
      ld16(5 * kAccStride + c, b);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int t = 0; t < 16; t++) im[t] = __uint_as_float(a[t]) + __uint_as_float(b[t]);
      if (!first) {
        ld16(kSumRe + c, a);
        ld16(kSumIm + c, b);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int t = 0; t < 16; t++) {
          re[t] = __uint_as_float(a[t]) + re[t];
          im[t] = __uint_as_float(b[t]) + im[t];
        }
      }
      st16(kSumRe + c, re);
      st16(kSumIm + c, im);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
  };

  auto arrive = [&](uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
  };
  // converter warps: lane 0 waits, the warp shares the outcome (warp-uniform)
  auto warp_wait = [&](void* bar, uint32_t parity) {
    int okw = 0;
    if (lane == 0) okw = mbar_wait(bar, parity, wait_ns) ? 1 : 0;
    okw = __shfl_sync(0xffffffffu, okw, 0);
    __syncwarp();
    return okw != 0;
  };
  // converter warps: every lane's shared-memory writes, then one arrival
  auto warp_arrive = [&](uint64_t* bar) {
    __syncwarp();
    if (lane == 0) arrive(bar);
  };
  if (warp < kConvWarps) {
    // converter group grp: its k-blocks kb = grp (mod kGroups), raw ring ->
    // TF32 planes of stage kb % kStages; the group that converts a chunk's
    // last k-block then moves the chunk's TMEM accumulators into the FP32 sums
    for (int kb = grp; kb < nkb; kb += kGroups) {
      const int stage = kb % kStages, slot = kb % kRing;
      // decisions are warp-uniform: the TMEM reads below are warp-collective
      if (__any_sync(0xffffffffu, !s_ok)) break;
      if (kb >= kStages &&
          !warp_wait(&empty[stage], (uint32_t)(((kb - kStages) / kStages) & 1))) {
        s_ok = 0;
        break;
      }
      if (!warp_wait(&raw_full[slot], (uint32_t)((kb / kRing) & 1))) {  // block kb landed
        s_ok = 0;
        break;
      }
      store(stage, kb);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
      warp_arrive(&full[stage]);
      warp_arrive(&raw_empty[slot]);  // the slot may take block kb + kRing
      if (kb % kChunk == kChunk - 1 || kb == nkb - 1) {
        // this group converted the chunk's last k-block: its four warps (one
        // per TMEM lane quarter) read the chunk out, all 64 columns each
        const int c = kb / kChunk;
        if (!warp_wait(&cdone[c & 1], (uint32_t)((c >> 1) & 1))) {
          s_ok = 0;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        flush(c == 0, 0, BN);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        warp_arrive(&flushed);  // the accumulators may be overwritten
      }
    }
  } else if (warp == kConvWarps + 1) {
    // TMA producer (lane 0): k-block kb into ring slot kb % kRing once the
    // converters have read the block before it in that slot
    if (lane == 0) {
      int last[kRing];
      for (int r = 0; r < kRing; r++) last[r] = -1;
      for (int kb = 0; kb < nkb; kb++) {
        const int slot = kb % kRing;
        if (!s_ok) break;
        if (kb >= kRing && !mbar_wait(&raw_empty[slot], (uint32_t)(((kb - kRing) / kRing) & 1), wait_ns)) {
          s_ok = 0;
          break;
        }
        unsigned char* dst = raw + slot * (kRawX + kRawY);
        mbar_expect_tx(&raw_full[slot], (uint32_t)(kRawX + kRawY));
        tma_load_3d(dst, &tmx, kb * 2 * BK, i0, (int)blockIdx.z, &raw_full[slot]);
        tma_load_3d(dst + kRawX, &tmy, kb * 2 * BK, j0, (int)blockIdx.z, &raw_full[slot]);
        last[slot] = kb;
      }
      // every load issued has landed before the CTA may exit (bounded, always
      // the full bound; one load per slot at most is outstanding)
      for (int r = 0; r < kRing; r++)
        if (last[r] >= 0 && !mbar_wait(&raw_full[r], (uint32_t)((last[r] / kRing) & 1), (uint64_t)kCgemmWaitNs))
          s_ok = 0;
    }
  } else if (lane == 0) {
    // tensor-core issuer
    for (int kb = 0; kb < nkb; kb++) {
      const int stage = kb % kStages, c = kb / kChunk;
      if (!s_ok) break;
      if (kb % kChunk == 0 && c > 0 && !mbar_wait(&flushed, (uint32_t)((c - 1) & 1), wait_ns)) {
        s_ok = 0;
        break;
      }
      if (!mbar_wait(&full[stage], (uint32_t)((kb / kStages) & 1), wait_ns)) {
        s_ok = 0;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sb = smem_u32(smem + stage * kStageBytes);
      const uint64_t xrh = smem_desc(sb + 0 * kXPlane), xrl = smem_desc(sb + 1 * kXPlane);
      const uint64_t xih = smem_desc(sb + 2 * kXPlane), xil = smem_desc(sb + 3 * kXPlane);
      const uint32_t yo = sb + 4 * kXPlane;
      const uint64_t yrh = smem_desc(yo + 0 * kYPlane), yrl = smem_desc(yo + 1 * kYPlane);
      const uint64_t yih = smem_desc(yo + 2 * kYPlane), yil = smem_desc(yo + 3 * kYPlane);
      const uint32_t acc = (kb % kChunk) ? 1u : 0u;  // a chunk starts from zero
      const uint32_t mp = tmem, mn = tmem + kAccStride, mi = tmem + 2 * kAccStride;
      const uint32_t cp = tmem + 3 * kAccStride, cn = tmem + 4 * kAccStride, ci = tmem + 5 * kAccStride;
      mma_tf32(mp, xrh, yrh, acc);  // Re+ = Xr Yr
      mma_tf32(cp, xrh, yrl, acc);
      mma_tf32(cp, xrl, yrh, 1u);
      mma_tf32(mn, xih, yih, acc);  // Re- = Xi Yi
      mma_tf32(cn, xih, yil, acc);
      mma_tf32(cn, xil, yih, 1u);
      mma_tf32(mi, xrh, yih, acc);  // Im = Xr Yi + Xi Yr
      mma_tf32(mi, xih, yrh, 1u);
      mma_tf32(ci, xrh, yil, acc);
      mma_tf32(ci, xrl, yih, 1u);
      mma_tf32(ci, xih, yrl, 1u);
      mma_tf32(ci, xil, yrh, 1u);
      mma_commit(&empty[stage]);
      if (kb % kChunk == kChunk - 1 || kb == nkb - 1) mma_commit(&cdone[c & 1]);
    }
    // everything issued has completed before TMEM is freed (bounded wait,
    // always the full bound)
    mma_commit(&fin);
    if (!mbar_wait(&fin, 0u, (uint64_t)kCgemmWaitNs)) s_ok = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (s_ok) {
    if (warp < kConvWarps) {  // the sums of this thread's row and 16 columns, TMEM -> HBM
      const int i = i0 + row;
      const uint32_t ibits = map.ld > 0 ? 0u : scat((uint32_t)i, map.ipos, map.ni);
      float2* ob = out + (int64_t)blockIdx.z * os;
      static_assert(kColW == 16, "one 16-column read per thread");
      uint32_t a[16], b[16];
      ld16(kSumRe + col0, a);
      ld16(kSumIm + col0, b);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int t = 0; t < 16; t++) {
        const int j = j0 + col0 + t;
        const float2 v = make_float2(__uint_as_float(a[t]), __uint_as_float(b[t]));
        if (map.ld > 0) ob[(int64_t)i * map.ld + j] = v;
        else ob[ibits | scat((uint32_t)j, map.jpos, map.nj)] = v;
      }
    }
  } else if (tid == 0) {
    atomicOr(status, 1 << TDQ_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kConvWarps) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

// cuTensorMapEncodeTiled, fetched from the driver once (no link to libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of an operand [batch][rows][K] complex64 (batch stride bs
// complex) as float [batch][rows][2K], boxes of 2 BK floats by box_rows rows.
static bool operand_map(CUtensorMap* m, const float2* base, int rows, int K, int64_t bs, int batch, int box_rows) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * K, (cuuint64_t)rows, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)K * 8, (cuuint64_t)(batch > 1 ? bs : (int64_t)rows * K) * 8};
  const cuuint32_t box[3] = {2 * BK, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t cgemm_tc_launch(const float2* X, int64_t xs, const float2* Y, int64_t ys, float2* out, int64_t os,
                            int I, int J, int K, int batch, const CgemmOut& map, int* status, cudaStream_t st,
                            const char** where, int64_t wait_ns) {
  if (I % BM || J % BN || K % BK || K <= 0 || batch < 1 || batch > 65535) {
    if (where) *where = "shape";
    return cudaErrorInvalidValue;
  }
  // TMA: operands on 16-byte boundaries, batch strides whole 16-byte units
  // that do not overlap the batch entry before (every box coordinate x =
  // 2 BK kb floats is a multiple of 16 bytes)
  if (((uintptr_t)X | (uintptr_t)Y) & 15u || (batch > 1 && ((xs & 1) || (ys & 1) || xs < (int64_t)I * K ||
                                                            ys < (int64_t)J * K))) {
    if (where) *where = "operand alignment";
    return cudaErrorInvalidValue;
  }
  CUtensorMap tmx, tmy;
  if (!operand_map(&tmx, X, I, K, xs, batch, BM) || !operand_map(&tmy, Y, J, K, ys, batch, BN)) {
    if (where) *where = "tensor map";
    return cudaErrorInvalidValue;
  }
  const cudaError_t e = cudaFuncSetAttribute(k_cgemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e != cudaSuccess) {
    if (where) *where = "shared-memory attribute";
    return e;
  }
  const dim3 grid((unsigned)(J / BN), (unsigned)(I / BM), (unsigned)batch);
  k_cgemm_tc<<<grid, kThreads, kSmemBytes, st>>>(tmx, tmy, out, os, K, map, status,
                                                 (uint64_t)(wait_ns > 0 ? wait_ns : 0));
  if (where) *where = "launch";
  return cudaGetLastError();
}

}  // namespace tdq

using namespace tdq;

// Kernel-level entry: row-major complex D[b] = X[b] Y[b]^T (see tdq.h).
extern "C" tdq_status tdq_cgemm_nt(int batch, int I, int J, int K, const float* dX, const float* dY, float* dD,
                                   int* d_status, void* stream) {
  return tdq_cgemm_nt_bounded(batch, I, J, K, dX, dY, dD, d_status, kCgemmWaitNs, stream);
}

extern "C" tdq_status tdq_cgemm_nt_bounded(int batch, int I, int J, int K, const float* dX, const float* dY,
                                           float* dD, int* d_status, int64_t wait_ns, void* stream) {
  if (wait_ns < 0 || wait_ns > kCgemmWaitNs)
    return fail(TDQ_ERR_ARG, "tdq_cgemm_nt_bounded: wait_ns must be in [0, 1e9]");
  if (!dX || !dY || !dD || !d_status) return fail(TDQ_ERR_ARG, "tdq_cgemm_nt: NULL argument");
  if (I <= 0 || J <= 0 || K <= 0 || I % 128 || J % 64 || K % 8 || batch < 1 || batch > 65535)
    return fail(TDQ_ERR_ARG, "tdq_cgemm_nt: need I % 128 == 0, J % 64 == 0, K % 8 == 0, 1 <= batch <= 65535");
  CgemmOut map{nullptr, nullptr, 0, 0, (int64_t)J};
  const cudaError_t e = cgemm_tc_launch(reinterpret_cast<const float2*>(dX), (int64_t)I * K,
                                        reinterpret_cast<const float2*>(dY), (int64_t)J * K,
                                        reinterpret_cast<float2*>(dD), (int64_t)I * J, I, J, K, batch, map, d_status,
                                        (cudaStream_t)stream, nullptr, wait_ns);
  if (e != cudaSuccess) return fail(TDQ_ERR_CUDA, std::string("tdq_cgemm_nt: ") + cudaGetErrorString(e));
  return ok();
}
