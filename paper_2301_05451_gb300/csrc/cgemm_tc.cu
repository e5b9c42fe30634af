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
// + warps kConvWarps .. kConvWarps + 3 (the flushers, one per TMEM lane
// quarter), kConvWarps + 4 (the tensor-core issuer), kConvWarps + 5 (the TMA
// producer)
constexpr int kFlushWarp0 = kConvWarps, kIssuerWarp = kConvWarps + 4, kProducerWarp = kConvWarps + 5;
constexpr int kThreads = kConv + 6 * 32;
static_assert(kFlushWarp0 % 4 == 0, "the flusher warps cover the four TMEM lane quarters");
// The converters work in kGroups groups of kGroupWarps warps; group g
// converts the k-blocks kb = g (mod kGroups), one whole k-block at a time, so
// that the groups' k-blocks are in flight together.  Per k-block a group
// thread converts one row of X (warp w of the group holds TMEM lanes 32 w ..,
// so that lane l takes row 32 w + l: four 16-byte loads, one per bank group
// under the raw ring's 128-byte swizzle, and one 32-column store of its four
// TF32 planes to TMEM) and kYP k-pairs of Y: lane l takes row 32 u + 8 w +
// (l % 8) and k-pair l / 8 for u = 0, 1, ... -- a quarter-warp reads eight
// rows of one k-pair and a half-warp writes one 8-row core matrix of a plane
// (8-byte stores, no bank conflict).
constexpr int kGroups = 4;
constexpr int kGroupWarps = kConvWarps / kGroups;
constexpr int kGroupThreads = kGroupWarps * 32;
constexpr int kYP = BN * BK / 2 / kGroupThreads;
static_assert(BK == 8 && kGroupWarps * 8 * 4 == kGroupThreads, "thread map: 8 rows x 4 k-pairs per warp");
static_assert(kGroupThreads == BM && kGroupWarps == 4, "one X row per group thread, four TMEM lane quarters");
static_assert(kYP * kGroupThreads == BN * BK / 2, "k-pairs per group thread");
// TMEM read-out in the epilogue: warp w reads lanes 32 (w % 4) .. and a group of kColW columns
constexpr int kColW = BN / (kConvWarps / 4);
constexpr int kYSub = BN * BK * 4;  // bytes: one real TF32 plane of the Y tile
// Y is stored as eight sub-planes of BN rows,
//   P, Q, P', Q', -Yi_P, Yr_P, -Yi_P', Yr_P'   with (P, Q) = (Yr, Yi),
// where P is the hi split and P' the lo split in a k-block of an even chunk,
// and the other way round in an odd chunk; so B1 = [Yr; Yi] (sub-planes 0-1
// or 2-3 for hi alone) and B2 = [-Yi; Yr] (4-5 or 6-7) are contiguous, and
// the 256-row operands [B_P; B_P'] (0-3, 4-7) put the hi rows first in an
// even chunk and last in an odd one.
constexpr int kYBytes = 8 * kYSub;
constexpr int kStageBytes = kYBytes;  // the Y planes (X's are in TMEM)
// TF32 plane stages in flight on the tensor cores, and raw operand slots in
// flight (TMA ring ahead of the split into planes).  A raw slot holds two
// k-blocks: TMA boxes of 128-byte rows (16 complex), half the row requests of
// one box per k-block, written with the 128-byte swizzle (the 16-byte chunk
// c of row r lands at chunk c ^ (r % 8)).  kStages >= kGroups and 2 kRing a
// multiple of kGroups: a converter's wait on a stage or a ring slot then
// never looks two phases back (the phase before is its own group's).
constexpr int kStages = 4;
constexpr int kRing = 4;
static_assert(kStages >= kGroups && (2 * kRing) % kGroups == 0, "pipeline depths");
constexpr int kRawX = BM * 2 * BK * 8, kRawY = BN * 2 * BK * 8;  // bytes of one raw slot (two complex k-blocks)
constexpr int kRawBytes = kRing * (kRawX + kRawY);
// FP32 sums of the flushed hi*hi chunks (round to nearest) in shared memory:
// 128 real columns (Re 0..63, Im 64..127) of 128 rows as float4 [col / 4][row],
// so that a thread (one row) reads and writes four columns at a time and a
// warp's 32 rows are 512 contiguous bytes.
constexpr int kSumBytes = 2 * BN * BM * 4;
// Shared memory per CTA: the Y plane stages, the raw ring and the sums.  It
// is above half the SM's shared memory, so one CTA runs per SM -- it then
// owns all 512 TMEM columns and tcgen05.alloc never waits for another CTA.
constexpr int kSmemBytes = kStages * kStageBytes + kRawBytes + kSumBytes;
static_assert(kSmemBytes <= 227 * 1024 - 512, "K3 shared memory");
static_assert(kSmemBytes > 114 * 1024, "K3: one CTA per SM");
constexpr uint32_t kTmemCols = 512;
// TMEM columns (128 lanes = the tile's rows):
//   0..127    hi*hi terms of an even chunk: Re (0..63), Im (64..127)
//   128..255  hi*lo + lo*hi correction terms of the whole K: Re, Im
//   256..383  hi*hi terms of an odd chunk: Re, Im
//   384..511  the products' A operand (X) of the kStages stages, 32 columns
//             each: Xr_hi, Xr_lo, Xi_hi, Xi_lo, 8 TF32 columns (k) apiece
// (X in TMEM keeps its planes off the shared memory, which the Y planes, the
// raw ring and the products' B operands share.)
// A 256-column product of an even chunk writes 0..255 (hi rows first), of an
// odd chunk 128..383 (lo rows first); the corrections are never flushed
// (they are 2^-11 of the hi*hi terms, so FP32 accumulation over any K keeps
// them far below the result's rounding), while the hi*hi chunks are
// accumulated alternately and flushed by dedicated warps, so the tensor cores
// never wait for a read-out.
constexpr uint32_t kCo = 128, kA = 384;
// The epilogue's staging tile: the 128 x 64 complex results, rows kStgLd
// complex apart (528 bytes: a quarter-warp's 16-byte stores of eight rows
// fall in distinct banks), over the plane stages and the raw ring.
constexpr int kStgLd = BN + 2;
static_assert(BM * kStgLd * 8 <= kStages * kStageBytes + kRawBytes, "epilogue staging tile");
static_assert((kStgLd * 8) % 16 == 0, "16-byte aligned staging rows");
constexpr int kChunk = 16;  // k-blocks of hi*hi terms accumulated in TMEM before a flush
static_assert(kA + 32 * kStages <= kTmemCols, "TMEM columns");

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
constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}
// Wide products do more work per cycle of the tensor pipe: issued back to
// back from one thread on GB300, an N = 64 product took about 48 cycles and
// an N = 256 one about 128 (a k-block of twelve N 64 products 577 cycles, of
// the four below 385), so the product is cut into as few, as wide,
// instructions as the accumulators allow.
constexpr uint32_t kIdesc256 = idesc_tf32(4 * BN), kIdesc128 = idesc_tf32(2 * BN);

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// One product D (+)= A B^T of kind::tf32 with A in TMEM (M rows in lanes, K
// TF32 in consecutive columns) and B in shared memory (descriptor); acc = 0
// starts D from zero.
__device__ __forceinline__ void mma_tf32_ta(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(acc));
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
  if (limit_ns == 0) return false;  // a zero bound: no waiting (the global timer is coarser than a poll)
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

__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 16 consecutive TMEM columns of this warp's 32 lanes -> registers
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// 32 consecutive TMEM columns of this warp's 32 lanes <- registers
__device__ __forceinline__ void st32(uint32_t taddr, const float (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]),
      "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]),
      "f"(v[16]), "f"(v[17]), "f"(v[18]), "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]),
      "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]), "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
      : "memory");
}

// X, Y: tensor maps over the operands as float [batch][rows][2K] (re, im
// interleaved), boxes of 2 BK complex by BM (X) / BN (Y) rows, 128-byte swizzle.
__global__ void __launch_bounds__(kThreads, 1)
    k_cgemm_tc(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmy, float2* out,
               int64_t os, int K, CgemmOut map, int* status, uint64_t wait_ns) {
  // wait for the kernel before this one in the stream (a launch with
  // programmatic stream serialisation may start early; otherwise this returns
  // at once), then let the next one be dispatched while this one runs
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ __align__(1024) unsigned char smem[];
  // full[s]: a converter group wrote stage s (one arrival per warp of the group);
  // empty[s]: the tensor cores are done with it (commit);
  // raw_full[r]: the TMA load of ring slot r landed (byte count); raw_empty[r]:
  // the converters read it (one arrival per converter warp of the two groups
  // whose k-blocks it holds);
  // cdone[c & 1]: the products of chunk c are in TMEM (commit); flushed[c & 1]:
  // the flushers moved chunk c's hi*hi terms into the sums (one arrival per
  // flusher warp); fin: every product issued has completed (commit).
  // A chunk's barriers alternate by its parity: chunk c + 2 reuses chunk c's
  // barrier only after chunk c was flushed, so no parity wait looks two
  // phases back.
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], cdone[2], flushed[2], fin;
  __shared__ __align__(8) uint64_t raw_full[kRing], raw_empty[kRing];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const int nkb = K / BK, nchunk = (nkb + kChunk - 1) / kChunk;

  if (tid == 0) {
    for (int s = 0; s < kStages; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(kGroupWarps));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
    }
    for (int p = 0; p < 2; p++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&cdone[p])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&flushed[p])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fin)));
    for (int r = 0; r < kRing; r++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&raw_full[r])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&raw_empty[r])), "r"(2 * kGroupWarps));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
  }
  if (warp == kIssuerWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t lane_addr = (uint32_t)((warp & 3) * 32) << 16;  // this warp's TMEM lane quarter
  unsigned char* raw = smem + kStages * kStageBytes;
  unsigned char* sumb = raw + kRawBytes;  // the FP32 sums (float4 [col / 4][row])

  // Every role runs warp-wide and stays converged: all lanes poll a wait
  // (the outcome made warp-uniform, as the TMEM accesses and the single-lane
  // issues after it need), one lane issues TMA loads, products and commits.
  // A lane left to loop alone while its warp waits at the final barrier made
  // the issuer several times slower than its products.
  auto warp_wait_for = [&](void* bar, uint32_t parity, uint64_t limit) {
    const bool okl = mbar_wait(bar, parity, limit);
    return __all_sync(0xffffffffu, okl);
  };
  auto warp_wait = [&](void* bar, uint32_t parity) { return warp_wait_for(bar, parity, wait_ns); };
  // every lane's shared-memory accesses, then one arrival for the warp
  auto warp_arrive = [&](uint64_t* bar) {
    __syncwarp();
    if (lane == 0) arrive(bar);
  };

  if (warp < kConvWarps) {
    // converter group grp: its k-blocks kb = grp (mod kGroups), raw ring ->
    // TF32 planes of stage kb % kStages.  Raw ring slot r holds the TMA boxes
    // of k-blocks 2 m and 2 m + 1, X [BM rows][2 BK complex] then Y [BN
    // rows][2 BK complex], 128 bytes a row, swizzled.  This thread converts
    // X row xr (its TMEM lane) and Y rows 32 u + rsub (u < kYP) at k-pair
    // kp, the plane offsets fixed per thread.
    const int grp = warp / kGroupWarps, gw = warp % kGroupWarps;
    const int rsub = 8 * gw + (lane & 7), kp = lane >> 3, xr = 32 * gw + lane;
    uint32_t yoff[kYP];
#pragma unroll
    for (int u = 0; u < kYP; u++) yoff[u] = plane_off(32 * u + rsub, 2 * kp);
    for (int kb = grp; kb < nkb; kb += kGroups) {
      const int stage = kb % kStages, pair = kb >> 1, slot = pair % kRing;
      if (__any_sync(0xffffffffu, !s_ok)) break;
      if (kb >= kStages && !warp_wait(&empty[stage], (uint32_t)(((kb - kStages) / kStages) & 1))) {
        s_ok = 0;
        break;
      }
      if (!warp_wait(&raw_full[slot], (uint32_t)((pair / kRing) & 1))) {  // block kb landed
        s_ok = 0;
        break;
      }
      unsigned char* base = smem + stage * kStageBytes;
      const float4* rx = reinterpret_cast<const float4*>(raw + slot * (kRawX + kRawY));
      const float4* ry = reinterpret_cast<const float4*>(raw + slot * (kRawX + kRawY) + kRawX);
      // 16-byte chunk of (row r, k-pair kp) of this k-block in a swizzled row
      const int h4 = 4 * (kb & 1), c0 = h4 + kp;
      float4 vx[4], vy[kYP];  // all loads first: one latency for the k-block
#pragma unroll
      for (int q = 0; q < 4; q++) vx[q] = rx[8 * xr + ((h4 + q) ^ (xr & 7))];
#pragma unroll
      for (int u = 0; u < kYP; u++) {
        const int r = 32 * u + rsub;
        vy[u] = ry[8 * r + (c0 ^ (r & 7))];
      }
      warp_arrive(&raw_empty[slot]);  // the values are in registers: the slot may take blocks 2 (m + kRing) ..
      // X: hi / lo TF32 split of the row's 8 complex values into the stage's
      // TMEM columns Xr_hi[k], Xr_lo[k], Xi_hi[k], Xi_lo[k] (k = 0..7); the
      // stage's earlier products are complete (the "empty" wait above)
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      {
        float xa[32];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const float re[2] = {vx[q].x, vx[q].z}, im[2] = {vx[q].y, vx[q].w};
#pragma unroll
          for (int t = 0; t < 2; t++) {
            const int k = 2 * q + t;
            const float rh = tf32_rna(re[t]), ih = tf32_rna(im[t]);
            xa[k] = rh;
            xa[8 + k] = tf32_rna(re[t] - rh);
            xa[16 + k] = ih;
            xa[24 + k] = tf32_rna(im[t] - ih);
          }
        }
        st32(tmem + ((uint32_t)(32 * gw) << 16) + kA + 32u * (uint32_t)stage, xa);
      }
      // Y: the same split into the eight sub-planes; hi first in an even
      // chunk, lo first in an odd one (the negated planes are exact: the
      // split commutes with the sign)
      const bool odd = ((kb / kChunk) & 1) != 0;
#pragma unroll
      for (int u = 0; u < kYP; u++) {
        const float4 v = vy[u];
        const float rh0 = tf32_rna(v.x), ih0 = tf32_rna(v.y), rh1 = tf32_rna(v.z), ih1 = tf32_rna(v.w);
        const float2 rh = make_float2(rh0, rh1), ih = make_float2(ih0, ih1);
        const float2 rl = make_float2(tf32_rna(v.x - rh0), tf32_rna(v.z - rh1));
        const float2 il = make_float2(tf32_rna(v.y - ih0), tf32_rna(v.w - ih1));
        const float2 rp = odd ? rl : rh, ip = odd ? il : ih, rq = odd ? rh : rl, iq = odd ? ih : il;
        unsigned char* p = base + yoff[u];
        *reinterpret_cast<float2*>(p + 0 * kYSub) = rp;
        *reinterpret_cast<float2*>(p + 1 * kYSub) = ip;
        *reinterpret_cast<float2*>(p + 2 * kYSub) = rq;
        *reinterpret_cast<float2*>(p + 3 * kYSub) = iq;
        *reinterpret_cast<float2*>(p + 4 * kYSub) = make_float2(-ip.x, -ip.y);
        *reinterpret_cast<float2*>(p + 5 * kYSub) = rp;
        *reinterpret_cast<float2*>(p + 6 * kYSub) = make_float2(-iq.x, -iq.y);
        *reinterpret_cast<float2*>(p + 7 * kYSub) = rq;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");   // the X planes are in TMEM
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      warp_arrive(&full[stage]);
    }
  } else if (warp < kIssuerWarp) {
    // flusher warp (TMEM lane quarter warp % 4, all of the tile's columns):
    // chunk c's hi*hi terms -> registers -> FP32 sums in shared memory
    // (round to nearest); this thread owns row `row` of the sums
    const int row = (warp & 3) * 32 + lane;
    float4* sums = reinterpret_cast<float4*>(sumb);
    for (int c = 0; c < nchunk; c++) {
      if (__any_sync(0xffffffffu, !s_ok)) break;
      if (!warp_wait(&cdone[c & 1], (uint32_t)((c >> 1) & 1))) {
        s_ok = 0;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t hh = tmem + lane_addr + ((c & 1) ? 256u : 0u);
#pragma unroll 1
      for (uint32_t col = 0; col < 2 * BN; col += 32) {
        uint32_t a[16], b[16];
        ld16(hh + col, a);
        ld16(hh + col + 16, b);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int t = 0; t < 8; t++) {
          const uint32_t* src = t < 4 ? a + 4 * t : b + 4 * (t - 4);
          float4* dst = sums + (size_t)((col >> 2) + t) * BM + row;
          float4 v = make_float4(__uint_as_float(src[0]), __uint_as_float(src[1]), __uint_as_float(src[2]),
                                 __uint_as_float(src[3]));
          if (c > 0) {
            const float4 o = *dst;
            v = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
          }
          *dst = v;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      warp_arrive(&flushed[c & 1]);  // the chunk's hi*hi columns may be overwritten
    }
  } else if (warp == kProducerWarp) {
    // TMA producer: k-blocks 2 m, 2 m + 1 into ring slot m % kRing once the
    // converters have read the pair before them in that slot (a last odd
    // k-block's box reads past K: TMA fills zeros there, never converted)
    const int npair = (nkb + 1) >> 1;
    int issued = 0;  // pairs whose loads were issued
    for (int m = 0; m < npair; m++) {
      const int slot = m % kRing;
      if (__any_sync(0xffffffffu, !s_ok)) break;
      if (m >= kRing && !warp_wait(&raw_empty[slot], (uint32_t)(((m - kRing) / kRing) & 1))) {
        s_ok = 0;
        break;
      }
      if (lane == 0) {
        unsigned char* dst = raw + slot * (kRawX + kRawY);
        mbar_expect_tx(&raw_full[slot], (uint32_t)(kRawX + kRawY));
        tma_load_3d(dst, &tmx, m * 4 * BK, i0, (int)blockIdx.z, &raw_full[slot]);
        tma_load_3d(dst + kRawX, &tmy, m * 4 * BK, j0, (int)blockIdx.z, &raw_full[slot]);
      }
      __syncwarp();
      issued = m + 1;
    }
    // every load issued has landed before the CTA may exit (bounded, always
    // the full bound; one load per slot at most is outstanding: the last
    // kRing pairs issued)
    for (int m = issued > kRing ? issued - kRing : 0; m < issued; m++)
      if (!warp_wait_for(&raw_full[m % kRing], (uint32_t)((m / kRing) & 1), (uint64_t)kCgemmWaitNs)) s_ok = 0;
  } else {
    // tensor-core issuer (lane 0 issues, the warp waits).  The k-block's
    // products, with the stage's "empty" commit and at a chunk's end the
    // "cdone" one:
    auto issue = [&](int kb) {
      const int stage = kb % kStages, c = kb / kChunk;
      const uint32_t sb = smem_u32(smem + stage * kStageBytes);
      // A (X) in TMEM: the stage's columns Xr_hi, Xr_lo, Xi_hi, Xi_lo
      const uint32_t xa = tmem + kA + 32u * (uint32_t)stage;
      const uint32_t xrh = xa, xrl = xa + 8u, xih = xa + 16u, xil = xa + 24u;
      const uint32_t yo = sb;
      const bool odd = (c & 1) != 0;
      // sub-planes of Y (see kYBytes): hi rows of B1 / B2 at yh / yh + 4,
      // lo rows at yl / yl + 4; the 256-row operands start at 0 / 4
      const uint32_t yh = odd ? 2u : 0u, yl = 2u - yh;
      const uint64_t b1 = smem_desc(yo), b2 = smem_desc(yo + 4 * kYSub);
      const uint64_t b1h = smem_desc(yo + yh * kYSub), b2h = smem_desc(yo + (4 + yh) * kYSub);
      // D of a 256-column product: hi*hi columns then corrections (even
      // chunk), or corrections then hi*hi columns (odd chunk)
      const uint32_t dw = tmem + (odd ? kCo : 0u), hh = tmem + (odd ? 256u : 0u), co = tmem + kCo;
      if (kb == 0) {
        mma_tf32_ta(dw, xrh, b1, kIdesc256, 0u);  // hi*hi and corrections start from zero
      } else if (kb % kChunk == 0) {
        // a new hi*hi chunk starts from zero; the corrections go on
        mma_tf32_ta(hh, xrh, b1h, kIdesc128, 0u);
        mma_tf32_ta(co, xrh, smem_desc(yo + yl * kYSub), kIdesc128, 1u);
      } else {
        mma_tf32_ta(dw, xrh, b1, kIdesc256, 1u);
      }
      // Re = Xr Yr - Xi Yi and Im = Xr Yi + Xi Yr side by side:
      //   Xr_hi [B1_hi; B1_lo] (above) + Xr_lo B1_hi + Xi_hi [B2_hi; B2_lo] + Xi_lo B2_hi
      mma_tf32_ta(co, xrl, b1h, kIdesc128, 1u);
      mma_tf32_ta(dw, xih, b2, kIdesc256, 1u);
      mma_tf32_ta(co, xil, b2h, kIdesc128, 1u);
      mma_commit(&empty[stage]);
      if (kb % kChunk == kChunk - 1 || kb == nkb - 1) mma_commit(&cdone[c & 1]);
    };
    // Two k-blocks per iteration: the loop's fixed cost (waits, fence,
    // convergence) measured about 360 cycles, most of a k-block's products,
    // so it is paid once per pair (a pair never straddles a chunk: kChunk is
    // even).  The cancellation flag is read once per chunk; every wait is
    // bounded on its own.
    static_assert(kChunk % 2 == 0, "k-block pairs within a chunk");
    for (int kb = 0; kb < nkb; kb += 2) {
      const int c = kb / kChunk;
      if (kb % kChunk == 0) {
        if (__any_sync(0xffffffffu, !s_ok)) break;
        // chunk c reuses the hi*hi columns of chunk c - 2: wait for its flush
        if (c >= 2 && !warp_wait(&flushed[c & 1], (uint32_t)(((c - 2) >> 1) & 1))) {
          s_ok = 0;
          break;
        }
      }
      const bool two = kb + 1 < nkb;
      if (!warp_wait(&full[kb % kStages], (uint32_t)((kb / kStages) & 1)) ||
          (two && !warp_wait(&full[(kb + 1) % kStages], (uint32_t)(((kb + 1) / kStages) & 1)))) {
        s_ok = 0;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (lane == 0) {
        issue(kb);
        if (two) issue(kb + 1);
      }
      __syncwarp();
    }
    // everything issued has completed before TMEM is freed (bounded wait,
    // always the full bound)
    if (lane == 0) mma_commit(&fin);
    __syncwarp();
    if (!warp_wait_for(&fin, 0u, (uint64_t)kCgemmWaitNs)) s_ok = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (s_ok && warp < kConvWarps) {
    // sums + corrections of this thread's row and 16 columns (TMEM lane =
    // row) into a staging tile in shared memory, free now that every product
    // and copy is complete; then each warp writes whole rows, lane l columns
    // 2 l and 2 l + 1, so that a store instruction covers 512 contiguous
    // bytes of a row-major result instead of one element of 32 rows
    const int row = (warp & 3) * 32 + lane, col0 = (warp >> 2) * kColW;
    static_assert(kColW == 16, "one 16-column read per thread");
    const uint32_t t = tmem + lane_addr;
    uint32_t cr[16], ci[16];
    ld16(t + kCo + col0, cr);
    ld16(t + kCo + BN + col0, ci);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const float4* sums = reinterpret_cast<const float4*>(sumb);  // float4 [col / 4][row]
    float4* srow = reinterpret_cast<float4*>(smem + (size_t)row * kStgLd * 8 + (size_t)col0 * 8);
#pragma unroll
    for (int q = 0; q < kColW / 4; q++) {
      const float4 sr = sums[(size_t)(col0 / 4 + q) * BM + row], si = sums[(size_t)((BN + col0) / 4 + q) * BM + row];
      const int u = 4 * q;
      srow[2 * q] = make_float4(sr.x + __uint_as_float(cr[u]), si.x + __uint_as_float(ci[u]),
                                sr.y + __uint_as_float(cr[u + 1]), si.y + __uint_as_float(ci[u + 1]));
      srow[2 * q + 1] = make_float4(sr.z + __uint_as_float(cr[u + 2]), si.z + __uint_as_float(ci[u + 2]),
                                    sr.w + __uint_as_float(cr[u + 3]), si.w + __uint_as_float(ci[u + 3]));
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kConv) : "memory");  // the converter warps only
    float2* ob = out + (int64_t)blockIdx.z * os;
    const int j = j0 + 2 * lane;
    const uint32_t jb0 = map.ld > 0 ? 0u : scat((uint32_t)j, map.jpos, map.nj);
    const uint32_t jb1 = map.ld > 0 ? 0u : scat((uint32_t)(j + 1), map.jpos, map.nj);
    for (int r = warp; r < BM; r += kConvWarps) {
      const float4 v = reinterpret_cast<const float4*>(smem + (size_t)r * kStgLd * 8)[lane];
      const int i = i0 + r;
      if (map.ld > 0) {
        float2* p = ob + (int64_t)i * map.ld + j;
        if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
          *reinterpret_cast<float4*>(p) = v;
        } else {
          p[0] = make_float2(v.x, v.y);
          p[1] = make_float2(v.z, v.w);
        }
      } else {
        const uint32_t ib = scat((uint32_t)i, map.ipos, map.ni);
        ob[ib | jb0] = make_float2(v.x, v.y);
        ob[ib | jb1] = make_float2(v.z, v.w);
      }
    }
  } else if (!s_ok && tid == 0) {
    atomicOr(status, 1 << TDQ_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kIssuerWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
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
// complex) as float [batch][rows][2K], boxes of 4 BK floats (two k-blocks,
// 128 bytes) by box_rows rows, written to shared memory with the 128-byte
// swizzle.
static bool operand_map(CUtensorMap* m, const float2* base, int rows, int K, int64_t bs, int batch, int box_rows) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * K, (cuuint64_t)rows, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)K * 8, (cuuint64_t)(batch > 1 ? bs : (int64_t)rows * K) * 8};
  const cuuint32_t box[3] = {4 * BK, (cuuint32_t)box_rows, 1};  // 16 complex: 128 bytes a row
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
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
  // programmatic stream serialisation: dispatched while the kernel before it
  // in the stream finishes; the kernel waits for it before any memory access
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(J / BN), (unsigned)(I / BM), (unsigned)batch);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kSmemBytes;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t le =
      cudaLaunchKernelEx(&cfg, k_cgemm_tc, tmx, tmy, out, os, K, map, status, (uint64_t)(wait_ns > 0 ? wait_ns : 0));
  if (where) *where = "launch";
  return le != cudaSuccess ? le : cudaGetLastError();
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
