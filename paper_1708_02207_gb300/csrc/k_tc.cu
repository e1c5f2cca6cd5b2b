// Schur-complement update on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// S -= X X^T over the b boundary rows of the large FP32 fronts (X = F[m:nf, 0:m];
// the bordered right-hand-side row is done by k_syrk_rhs), i.e. the SYRK of the
// partial Cholesky of Sec. 2.4
// (Eq. SchurC1: A11 - A12 A22^-1 A21 = K_BB - L_Bg L_Bg^T).  One CTA of 128
// threads computes one 128 x 64 tile (rows TI, columns TJ, on or below the
// diagonal) of one (node, sample):
//   * the TRSM that produced X also wrote it split into TF32 hi and lo parts,
//     in 128-row x 8-column tiles in the K-major, no-swizzle core-matrix layout
//     (8-row x 16-byte core matrices) that the MMA reads from shared memory;
//   * one thread runs the pipeline: TMA copies (cp.async.bulk.tensor through two
//     tensor maps over the batch's staging arena, viewed as rows of 1 KiB:
//     8-row boxes for an A tile's hi and lo parts, 2-row boxes for a B half;
//     completion counted in bytes on an mbarrier) fill kStages shared-memory
//     stages (launches over several plans, whose arenas differ, use plain
//     cp.async.bulk copies of the same bytes), and for each
//     8-column chunk it issues tcgen05.mma kind::tf32 (M = 128, N = 64, K = 8)
//     three times per step, hi*hi + hi*lo + lo*hi ("3xTF32", about FP32
//     accuracy), with the accumulator in tensor memory (128 lanes x 64 columns);
//     the B operand is one half (64 rows) of a 128-row staging tile;
//     tcgen05.commit frees a stage for the next copy;
//   * every wait is bounded (StepArgs::wait_limit polls); after a wait runs out
//     the thread issues no further copies or MMAs, waits (with the same bound)
//     for the MMAs already issued (one more tcgen05.commit on a drain barrier)
//     and for every copy already issued, and marks the sample HDD_ETIMEOUT; the
//     tensor memory is released only once no MMA can still write it;
//   * the four warps read their 32 accumulator lanes with tcgen05.ld, 16 columns at
//     a time, and subtract them from S (coalesced along the rows of S).
// The epilogue's gather of the sons' entries (Eq. block_equation4), a chain of
// dependent loads, bounds the kernel, so the tile is 128 x 64: eight CTAs of 64
// tensor-memory columns fill an SM's 512 columns and keep twice the warps of
// 128 x 128 tiles in flight on the gather.
#include <cuda.h>   // CUtensorMap (the encoder is taken from the driver at run time)

#include <mutex>

#include "launch.h"

namespace hdd {

namespace {

constexpr int kTile = kTcTile;        // M of the MMA: rows of the output tile
constexpr int kTileN = kTcTile / 2;   // N of the MMA: columns of the output tile
constexpr int kChunk = kTcChunk;      // contraction columns staged per buffer
constexpr int kTileBytes = (int)kTcBlockBytes;          // one operand part of 128 rows (4 KiB)
constexpr int kHalfBytes = kTileBytes / 2;              // its 64-row half (2 KiB)
constexpr int kStageBytes = 2 * kTileBytes + 2 * kHalfBytes;   // A hi/lo, B hi/lo (12 KiB)
// Pipeline depth: 2 stages (24 KiB).  The contraction is short (K = m = 31..511
// columns): the kernel wants CTAs in flight more than deep prefetch.
constexpr int kStages = 2;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle.  lbo = bytes between
// core matrices along K, sbo = bytes between 8-row groups; bit 46 = descriptor
// version of tcgen05.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, N = 64, M = 128.
__device__ __forceinline__ uint32_t idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mbar), "r"(phase));
    if (done) return true;
  }
  return false;
}

}  // namespace

// use_tma: the tensor maps describe this launch's staging arena (rows of 1 KiB from
// a.arenas.tc); otherwise the same bytes come by plain bulk copies.
__global__ void __launch_bounds__(128, 8) k_syrk_tc(StepArgs a, const __grid_constant__ CUtensorMap mapA,
                                                    const __grid_constant__ CUtensorMap mapB, int use_tma) {
  const int node = a.list[blockIdx.y];
  const int s = blockIdx.z;
  bind_plan(a, node);
  if (s >= a.batch) return;
  const NodeDev nd = a.nodes[node];
  const int m = nd.m, nb = nd.b + 1, nbt = nd.b;   // tiles cover the b boundary rows
  const int nt = (nbt + kTile - 1) / kTile;
  // row tile TI holds the column tiles TJ = 0 .. 2 TI + 1 (x = TI (TI + 1) + TJ)
  if ((int)blockIdx.x >= nt * (nt + 1) || m == 0 || nd.tc_off < 0) return;
  int TI = (int)((sqrtf(4.0f * (float)blockIdx.x + 1.0f) - 1.0f) * 0.5f);
  while (TI * (TI + 1) > (int)blockIdx.x) --TI;
  while ((TI + 1) * (TI + 2) <= (int)blockIdx.x) ++TI;
  const int TJ = blockIdx.x - TI * (TI + 1);
  if (TJ * kTileN >= nbt) return;   // columns beyond the boundary rows

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* stage =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int timed_out, mma_live;
  __shared__ int cpos[2][kTileN];   // sons' rows of this tile's columns (fathers)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTileN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int b = 0; b < kStages; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[b])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&drain)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    timed_out = 0;
    mma_live = 0;
  }
  const bool gather = !nd.leaf;
  const int32_t* pos0 = a.maps + nd.map_off + (nd.nf - 1);
  const int32_t* pos1 = pos0 + nd.nf;
  if (gather && tid < kTileN) {
    const int j = TJ * kTileN + tid;
    cpos[0][tid] = j < nbt ? pos0[m + j] : -1;
    cpos[1][tid] = j < nbt ? pos1[m + j] : -1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  // Epilogue operands.  The values subtracted from are loaded chunk by chunk
  // (32 columns), the first chunk before the MMAs so that its loads overlap
  // them.
  float* S = a.arenas.s32 + (int64_t)s * a.arenas.s32_stride + nd.s_off;
  const int i = TI * kTile + warp * 32 + lane;   // accumulator lane = tile row
  // fathers: the boundary block of the front is the sum of the sons' Schur
  // entries (Eq. block_equation4), gathered here (rows of one column are
  // consecutive in the son as in the father: both order boundary vertices
  // by id); leaves: their boundary block was filled into S
  NodeDev ch0{}, ch1{};
  const float *S0 = nullptr, *S1 = nullptr;
  int p0 = -1, p1 = -1;
  bool mixed_sons = false;
  if (gather) {
    ch0 = a.nodes[nd.child0];
    ch1 = a.nodes[nd.child1];
    mixed_sons = ch0.fp64 || ch1.fp64;
    S0 = a.arenas.s32 + (int64_t)s * a.arenas.s32_stride + ch0.s_off;
    S1 = a.arenas.s32 + (int64_t)s * a.arenas.s32_stride + ch1.s_off;
    if (i < nbt) {
      p0 = pos0[m + i];
      p1 = pos1[m + i];
    }
  }
  const int ld0 = ch0.b + 1, ld1 = ch1.b + 1;
  const int32_t* map = a.maps + nd.map_off;
  auto load_chunk = [&](int c0, float (&sv)[16]) {
    if (!gather) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int j = TJ * kTileN + c0 + q;
        sv[q] = (i < nbt && j < nbt && i >= j) ? S[(int64_t)j * nb + i] : 0.0f;
      }
    } else if (!mixed_sons) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int j = TJ * kTileN + c0 + q;
        const int q0 = cpos[0][c0 + q], q1 = cpos[1][c0 + q];
        const bool v = i < nbt && j < nbt && i >= j;
        float x = 0.0f;
        if (v && p0 >= 0 && q0 >= 0) x = S0[min(p0, q0) * ld0 + max(p0, q0)];
        if (v && p1 >= 0 && q1 >= 0) x += S1[min(p1, q1) * ld1 + max(p1, q1)];
        sv[q] = x;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int j = TJ * kTileN + c0 + q;
        sv[q] = (i < nbt && j < nbt && i >= j)
                    ? father_entry<float>(m + i, m + j, s, nd, map, ch0, ch1, a.arenas, a.rhs)
                    : 0.0f;
      }
    }
  };
  float sv[16];
  load_chunk(0, sv);

  if (tid == 0) {
    // one thread runs the pipeline: bulk copies of the split tiles (TI: A, TJ: B)
    // into kStages shared-memory stages, tensor-core MMAs out of them
    const int nchunks = (m + kChunk - 1) / kChunk;
    const unsigned char* base = a.arenas.tc + (int64_t)s * a.arenas.tc_stride + nd.tc_off;
    const uint32_t idesc = idesc_tf32();
    const uint32_t sbo = (kChunk / 4) * 128;
    const uint32_t limit = a.wait_limit;
    // test hook: the copies of one chunk of one (node, sample) are never issued, so
    // the wait for them runs out (the stage's barrier still expects their bytes)
    const int stall_chunk = (node == a.stall_node && s == a.stall_sample) ? min(1, nchunks - 1) : -1;
    uint32_t ph_full[kStages] = {}, ph_empty[kStages] = {};
    uint32_t pending = 0;   // bit b: copies into stage b issued, their completion not yet waited for
    bool ok = true, any_mma = false;
    // tensor-map rows (1 KiB each) of this (node, sample)'s staging
    const int row0 = (int)(((int64_t)s * a.arenas.tc_stride + nd.tc_off) >> 10);
    auto load = [&](int c) {
      const int b = c % kStages;
      const uint32_t dst = smem_u32(stage + b * kStageBytes);
      const uint32_t bar = smem_u32(&full[b]);
      const unsigned char* srcA = base + ((int64_t)TI * nchunks + c) * 2 * kTileBytes;
      // B: the half (TJ & 1) of the 128-row tile TJ / 2, hi part then lo part
      const unsigned char* srcB = base + ((int64_t)(TJ >> 1) * nchunks + c) * 2 * kTileBytes + (TJ & 1) * kHalfBytes;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kStageBytes));
      if (c == stall_chunk) return;
      if (use_tma) {
        const int ya = row0 + (TI * nchunks + c) * 8;
        const int yb = row0 + ((TJ >> 1) * nchunks + c) * 8 + (TJ & 1) * 2;
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
            ::"r"(dst), "l"(reinterpret_cast<uint64_t>(&mapA)), "r"(0), "r"(ya), "r"(bar)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
            ::"r"(dst + 2 * kTileBytes), "l"(reinterpret_cast<uint64_t>(&mapB)), "r"(0), "r"(yb), "r"(bar)
            : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
            ::"r"(dst + 2 * kTileBytes + kHalfBytes), "l"(reinterpret_cast<uint64_t>(&mapB)), "r"(0), "r"(yb + 4),
              "r"(bar)
            : "memory");
        pending |= 1u << b;
        return;
      }
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                   "l"(srcA), "r"(2 * kTileBytes), "r"(bar)
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       dst + 2 * kTileBytes),
                   "l"(srcB), "r"(kHalfBytes), "r"(bar)
                   : "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       dst + 2 * kTileBytes + kHalfBytes),
                   "l"(srcB + kTileBytes), "r"(kHalfBytes), "r"(bar)
                   : "memory");
      pending |= 1u << b;
    };
    for (int c = 0; c < nchunks && c < kStages; ++c) load(c);
    for (int c = 0; c < nchunks; ++c) {
      const int b = c % kStages;
      if (!mbar_wait(smem_u32(&full[b]), ph_full[b], limit)) { ok = false; break; }
      ph_full[b] ^= 1u;
      pending &= ~(1u << b);
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t Ah = smem_u32(stage + b * kStageBytes);
      const uint32_t Al = Ah + kTileBytes, Bh = Ah + 2 * kTileBytes, Bl = Bh + kHalfBytes;
#pragma unroll
      for (int t = 0; t < kChunk / 8; ++t) {
        const uint32_t o = t * 256;   // two core matrices (128 bytes apart along K) per MMA
        const uint64_t dah = smem_desc(Ah + o, 128, sbo), dal = smem_desc(Al + o, 128, sbo);
        const uint64_t dbh = smem_desc(Bh + o, 128, sbo), dbl = smem_desc(Bl + o, 128, sbo);
        mma_tf32(tmem, dah, dbh, idesc, (c > 0 || t > 0) ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, idesc, 1u);
        mma_tf32(tmem, dal, dbh, idesc, 1u);
      }
      any_mma = true;
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&empty[b])));
      // refill the stage of the previous chunk (its MMAs were queued one step
      // earlier), so that the MMAs of this chunk stay queued meanwhile
      const int cp = c - 1;
      if (cp >= 0 && cp + kStages < nchunks) {
        const int bp = cp % kStages;
        if (!mbar_wait(smem_u32(&empty[bp]), ph_empty[bp], limit)) { ok = false; break; }
        ph_empty[bp] ^= 1u;
        load(cp + kStages);
      }
    }
    // chunks whose commits have not been waited for: the last kStages, and the
    // last chunk when it had no refill step
    if (ok)
      for (int c = max(0, nchunks - kStages); c < nchunks; ++c) {
        const int b = c % kStages;
        if (!mbar_wait(smem_u32(&empty[b]), ph_empty[b], limit)) { ok = false; break; }
        ph_empty[b] ^= 1u;
      }
    if (!ok) {
      // Nothing more is issued.  A commit on the drain barrier completes once every
      // MMA this thread issued has completed; copies already issued complete on their
      // stage's barrier (a stage whose copies were never issued is not waited for).
      timed_out = 1;
      if (any_mma) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&drain)));
        if (!mbar_wait(smem_u32(&drain), 0u, limit)) mma_live = 1;
      }
      for (int b = 0; b < kStages; ++b)
        if (pending & (1u << b)) mbar_wait(smem_u32(&full[b]), ph_full[b], limit);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (timed_out) {
    if (tid == 0) flag_status(a.status, s, -HDD_ETIMEOUT, node);
  } else {
    const int row_last = TI * kTile + warp * 32 + 31;   // this warp's last row
#pragma unroll 1
    for (int c0 = 0; c0 < kTileN; c0 += 16) {
      if (TJ * kTileN + c0 > row_last) break;   // strictly above the diagonal of this warp's rows
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      if (c0 > 0) load_chunk(c0, sv);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int j = TJ * kTileN + c0 + q;
        if (i < nbt && j < nbt && i >= j) S[(int64_t)j * nb + i] = sv[q] - __uint_as_float(r[q]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  // an MMA that did not complete within the bound may still write this tensor
  // memory: it stays allocated rather than being handed to another CTA under it
  if (warp == 0 && !mma_live)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTileN));
}

constexpr size_t kSyrkTcSmem = kStages * (size_t)kStageBytes + 1024;

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
std::once_flag g_encode_once;

EncodeTiledFn encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  });
  return g_encode;
}

// A 2D FP32 tensor of rows of 256 values (1 KiB) over `rows` rows from `base`,
// read in boxes of 256 x box_rows.
bool encode_rows(CUtensorMap* map, void* base, uint64_t rows, uint32_t box_rows) {
  EncodeTiledFn enc = encoder();
  if (!enc || rows == 0 || rows > 0xFFFFFFFFull || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  const cuuint64_t dims[2] = {256, rows};
  const cuuint64_t strides[1] = {1024};
  const cuuint32_t box[2] = {256, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

cudaError_t launch_syrk_tc(const StepArgs& a, cudaStream_t st) {
  if (a.nlist == 0) return cudaSuccess;
  const int nt = (a.max_b + kTile - 1) / kTile;
  if (nt == 0) return cudaSuccess;
  dim3 grid(nt * (nt + 1), a.nlist, a.batch);
  // one plan: the staging arena of the batch as one tensor (row offsets of nodes and
  // samples are multiples of 8 KiB); several plans: plain bulk copies
  CUtensorMap mapA{}, mapB{};
  const uint64_t rows = (uint64_t)a.batch * (uint64_t)a.arenas.tc_stride / 1024;
  const bool tma = !a.plan_of && a.arenas.tc_stride % 1024 == 0 && encode_rows(&mapA, a.arenas.tc, rows, 8) &&
                   encode_rows(&mapB, a.arenas.tc, rows, 2);
  k_syrk_tc<<<grid, 128, kSyrkTcSmem, st>>>(a, mapA, mapB, tma ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t configure_tc_kernels() {
  return cudaFuncSetAttribute(k_syrk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSyrkTcSmem);
}

}  // namespace hdd
