// Tensor-core (tcgen05) lowerings of the SgemmLeaf node (Section 6.1) for
// sm_103a: the BF16x3 split tier, the plain BF16 tier and the block-scaled
// FP8 (E4M3) tier.
//
// The leaf computes C <- alpha*op(A)*op(B) + beta*C (column-major FP32, C
// not read when beta == 0). The paper computes in FP32 on CUDA cores; here
// each FP32 operand x is split into BF16 parts hi = bf16_rn(x) and
// lo = bf16_rn(x - hi) and the leaf sums the three products
// hi*hi + hi*lo + lo*hi on the tensor cores into one FP32 accumulator in
// tensor memory (the BF16 tier keeps hi*hi only; the FP8 tier multiplies
// E4M3 codes and scales each 128-wide K block by its two block scales).
// The BF16x6 tier splits each operand into three parts, hi, mid =
// bf16_rn(x - hi) and lo = bf16_rn(x - hi - mid), whose sum is x itself
// for every FP32 x away from the subnormal range, and sums the six
// products whose size is at least 2^-17 of hi*hi (lo*hi, hi*lo, mid*mid,
// mid*hi, hi*mid, hi*hi): the dropped ones are below 2^-25.
//
// Mapping of the dataflow graph (Section 3.4): one internal-node instance
// (an output tile) is one CTA (128 x 256) or a pair of CTAs in a cluster
// (256 x 256, cta_group::2); the Allocation node's tile memory is a ring of
// STAGES shared-memory slabs filled by TMA (the paper's scratchpad tiles),
// plus the accumulator tiles in tensor memory; the replicated leaf's
// multiply-accumulate is a sequence of tcgen05.mma instructions.
//
// Kernels
//   split_mmajor / split_kmajor / split_batch: FP32 op(X) -> K-major BF16
//       hi (and lo, and for BF16x6 a third) planes, rows of Kp =
//       roundup(K, 8) elements.
//   quant_fp8: FP32 op(X) -> E4M3 codes and one FP32 scale per 128 x 128
//       block.
//   sgemm_tc<MODE, EPI, GROUPED, PAIR, CONVERT>: persistent; warp 0 issues
//       TMA loads, warp 1 allocates tensor memory and issues the MMAs,
//       warps 2, 3 convert FP32 operands into planes (CONVERT), warps 4..11
//       read the accumulator (tcgen05.ld) into FP32 registers and write C
//       (with a merged elementwise leaf, EPI), and on request the BF16
//       planes of C a later leaf reads (forwarded to the next stage of a
//       multi-stage launch, or C's rows into the plane cache), with or
//       without C itself. A last round of tiles that would leave most units
//       idle runs in K halves whose partial sums meet in the workspace
//       (tail split). Every mbarrier wait is bounded; on expiry the kernel
//       sets a bit in the status word, drains its own copies and MMAs
//       (bounded again), frees tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/hpvm.h"
#include "internal.h"

namespace hpvm {
namespace {

constexpr int BM = 128;             // tile rows (M) = tensor-memory lanes
constexpr int BN = 256;             // tile columns (N) = accumulator columns
constexpr int EPI_WARPS = 8;        // two per tensor-memory lane quarter
constexpr int EPI_WARP0 = 4;        // warpgroup 0: producer, MMA, two idle warps
constexpr int THREADS = EPI_WARP0 * 32 + EPI_WARPS * 32;  // 3 warpgroups
// Register split (setmaxnreg): the block is launched with THREADS x
// LAUNCH_REGS registers (the cap __launch_bounds__(THREADS, 1) gives); the
// control warpgroup gives registers back and the two epilogue warpgroups,
// which hold a 128-column FP32 running sum per thread, take them.
constexpr int LAUNCH_REGS = 168;
// The split per leaf variant: ptxas's spills (-Xptxas -v) for 40/232 and
// 48/224 differ by variant, and each takes the one that spills least.
template <int MODE, int EPI, bool PAIR, bool CONVERT = false>
struct RegSplit {
  static constexpr int EPI_R = EPI == 2 ? 224 : 232;
  static constexpr int CTRL_R = EPI_R == 224 ? 48 : 40;
  static_assert(EPI_WARP0 * 32 * CTRL_R + EPI_WARPS * 32 * EPI_R <= THREADS * LAUNCH_REGS,
                "register split exceeds the launch's registers");
};
constexpr uint32_t TMEM_COLS = 2 * BN;        // all 512 columns: the FP32 chunk buffers
constexpr int GROUP_N = 8;          // column tiles per rasterisation group
constexpr uint32_t SMEM_BUDGET = 226 * 1024;  // of the 227 KB a block may have
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s per bounded wait
constexpr int FP8_BLOCK = 128;      // FP8 scale block (rows x K) of each operand

// status bits (DeviceStatus word)
constexpr int ST_PRODUCER = 1, ST_MMA = 2, ST_EPILOGUE = 4, ST_DRAIN = 8, ST_SELFTEST = 16, ST_CONFIG = 32,
              ST_CONVERT = 64;

// Leaf modes: 3 = BF16x3 split (hi*hi + hi*lo + lo*hi), 6 = BF16x6 (three
// BF16 parts per operand, six products), 1 = BF16, 8 = FP8 E4M3 with one
// FP32 scale per 128 x 128 block of each operand.
// PAIR: two CTAs of a cluster share one 256 x 256 tile (tcgen05 cta_group::2):
// each stages its own 128 rows of A and 128 of the tile's 256 rows of B, so
// per CTA a stage holds a third less and the operand traffic from L2 and the
// shared-memory reads of the MMAs drop by the same third.
template <int MODE, bool PAIR = false>
struct Cfg {
  static constexpr bool FP8 = MODE == 8;
  static constexpr int PLANES = MODE == 3 ? 2 : MODE == 6 ? 3 : 1;
  static constexpr int ELEM_BYTES = FP8 ? 1 : 2;
  // One K slab row in shared memory: 128 bytes (128-byte swizzle), so a
  // slab carries 4 K steps and the per-slab handshake is paid once per 4.
  // BF16x3 on a single CTA (batch policies 0-3) keeps 64-byte rows (64-byte swizzle):
  // its 4 planes of 384 rows would leave two 96 KiB stages; on a pair each
  // CTA stages 256 rows and three 64 KiB stages fit. BF16x6 (on pairs)
  // takes 64-byte rows: six 128-row planes per stage in four 48 KiB stages,
  // 2 K steps x 6 products = 12 MMAs per slab, as BF16x3 has per 128-byte
  // slab.
  static constexpr int ROW_BYTES = ((MODE == 3 && !PAIR) || MODE == 6) ? 64 : 128;
  static constexpr uint32_t A_SLAB = BM * ROW_BYTES;  // bytes of one A plane slab
  // Tile columns and tensor-memory buffers, and the split of a tile's
  // columns between the two epilogue warps of a lane quarter (multiples of
  // 32). Every leaf takes 256-column tiles in two buffers: narrower FP8
  // tiles in more buffers (128 x 4, 160 x 3, 192 x 2) measured 1.7-1.9x
  // slower at 8192, an MMA of N < 256 costing nearly as much as N = 256.
  static constexpr int TN = BN;
  static constexpr int NBUF = 2;
  static constexpr int COLS0 = TN / 2;
  static constexpr int COLS1 = TN - COLS0;
  static constexpr int ACC = COLS0 > COLS1 ? COLS0 : COLS1;
  static_assert(NBUF * TN <= (int)TMEM_COLS && COLS0 % 32 == 0 && COLS1 % 32 == 0, "tensor-memory buffers");
  static constexpr int B_ROWS = PAIR ? TN / 2 : TN;     // rows of B this CTA stages
  static constexpr uint32_t B_SLAB = B_ROWS * ROW_BYTES;  // bytes of one B plane slab
  static constexpr int BK = ROW_BYTES / ELEM_BYTES;   // K elements per slab
  static constexpr int MMA_K = 32 / ELEM_BYTES;           // K per tcgen05.mma
  // K chunk accumulated afresh in tensor memory and then added to FP32
  // registers with round-to-nearest (the tensor-core accumulation
  // truncates). BF16x3: 192 elements, whose 5e-6 bound the truncation over
  // a long K would break. At M = N = K = 8192 a model of the truncating
  // accumulation gives a normwise error of 4.50e-6 / 4.58e-6 / 4.94e-6 for
  // chunks of 128 / 256 / 512 (the BF16x3 floor is 4.39e-6); 192-element
  // chunks measured 4.48e-6 and a 3.7% faster leaf than 128 (two thirds as many
  // tensor-memory drains per K; longer chunks then wait on the TMA ring).
  // FP8: exactly one 128-element scale block, multiplied by its two block
  // scales when it is added. Plain BF16 (bound 1e-2) accumulates all of K
  // in tensor memory: one chunk per tile, read out once. BF16x6: 96
  // elements, 6 K steps x 6 products = 36 MMAs a chunk as BF16x3 has in 192
  // (the truncation grows with the MMAs a chunk accumulates, and the drains
  // per MMA stay as frequent).
  static constexpr int KC_SLABS = MODE == 1 ? (1 << 24) : (MODE == 3 ? 192 : MODE == 6 ? 96 : 128) / BK;
  static constexpr uint32_t STAGE_BYTES = PLANES * (A_SLAB + B_SLAB);
  static constexpr int STAGES = (int)((SMEM_BUDGET - 1536) / STAGE_BYTES) > 8
                                    ? 8 : (int)((SMEM_BUDGET - 1536) / STAGE_BYTES);
  static constexpr uint32_t SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 512 /*barriers*/;
  static_assert(2 * STAGES * 8 + 2 * NBUF * 8 + 8 <= 512, "barrier area");
  static_assert(MODE != 8 || KC_SLABS * BK == FP8_BLOCK, "FP8: one chunk per scale block");
  static_assert(MODE != 3 || KC_SLABS * BK == 192, "BF16x3: chunks of 192 K elements");
  static_assert(MODE != 6 || (KC_SLABS * BK == 96 && PAIR), "BF16x6: chunks of 96 K elements, on pairs");
};

// Kept within 120 bytes: ptxas spills the epilogue of the plain leaf once
// this struct grows past 128 (the two K-major row lengths are 32-bit and
// fill alignment gaps).
struct TcParams {
  int M, N, K;
  int row_kp;  // row planes: elements per plane row
  float* C;
  int64_t ldc;
  float alpha, beta;
  const float* scaleA;  // FP8: [ceil(M/128)][nkb] block scales of op(A)
  const float* scaleB;  // FP8: [ceil(N/128)][nkb] block scales of op(B)^T
  int nkb;              // FP8: ceil(K/128)
  int fwd_kp;           // forwarded planes: elements per plane row
  int* status;
  const float* aux;     // EPI 2: H, column-major with leading dimension ldaux
  int64_t ldaux;
  // Forwarded operand planes of C (or null): column n of C as K-major row n
  // (fwd_kp elements a row) of a BF16 hi plane and, BF16x3, a lo plane.
  __nv_bfloat16* fwd_hi;
  __nv_bfloat16* fwd_lo;
  // Row planes of C (or null): row m of C as K-major row m (row_kp
  // elements) of a BF16 hi plane and, BF16x3, of the lo plane that follows
  // it (the operand_layout(M, N) offsets), for a later leaf that reads C
  // with rows of C as operand rows (op(A) = A, op(B) = B^T).
  __nv_bfloat16* row_hi;
  // Tail split (or null): the partial sums of the K halves of the last
  // round's tiles, then one arrival counter per tile, CTA and epilogue warp
  // (zeroed before the launch).
  float* split_ws;
  // 1: C itself is not stored (only the planes of it this launch writes)
  int planes_only;
  // limit of each bounded wait in microseconds (0: WAIT_LIMIT_NS)
  uint32_t wait_limit_us;
};
static_assert(sizeof(TcParams) <= 128, "the leaf's parameters stay within 128 bytes");
__device__ __forceinline__ uint64_t wait_limit(const TcParams& p) {
  return p.wait_limit_us ? (uint64_t)p.wait_limit_us * 1000ull : WAIT_LIMIT_NS;
}

// In-leaf operand conversion (the BF16x3 leaf on pairs, op(A) and op(B)^T
// with their rows contiguous, as in the example's NT form): instead of two
// split launches before the leaf, the leaf's two idle control warps write
// the split planes. The operands are cut into chunks of 128 rows (one CTA's
// share of a pair tile) by one 64-element K slab; the warps of all CTAs
// take chunks from a global counter in the order the tiles first need them
// (the rounds of the grouped tile order; within a round, slab by slab
// across the round's row blocks), stage each chunk's FP32 values through
// shared memory in four TMA pieces of 32 rows, write the hi and lo planes,
// and release a per-chunk flag. The producer acquires the flags of the two
// chunks a slab reads before its TMA loads. Chunks are claimed only by
// running CTAs and converting one waits on nothing else, so every claimed
// chunk is finished; all waits are bounded. The first round's blocks, which
// every pair needs at once from the first slab on, are split by the split
// kernel before the launch (pre): converting them inside the leaf held its
// first round back (GB300, 8192: leaf 1.93-2.09 ms against 1.73-1.92 ms
// with every block ready), while the later rounds' blocks are converted
// long before they are read.
constexpr int CV_ROWS = 128;    // rows of a chunk
constexpr int CV_BK = 64;       // K elements of a chunk (the leaf's slab)
constexpr int CV_PIECE = 32;    // rows of a staged piece
constexpr int CV_PIECES = CV_ROWS / CV_PIECE;
constexpr uint32_t CV_PIECE_BYTES = CV_PIECE * CV_BK * 4;  // 8 KiB of FP32
constexpr int CV_WARPS = 2;     // warps 2 and 3
constexpr int CV_MAX_ROUNDS = 64;
constexpr int CV_TAB = 5;       // per round: A blocks [lo, hi), B blocks [lo, hi), first chunk
constexpr uint32_t CV_SMEM = CV_WARPS * 2 * CV_PIECE_BYTES + (CV_MAX_ROUNDS + 1) * CV_TAB * 4;
struct SplitOp;
struct SplitTile;
struct ConvParams {
  CUtensorMap src[2];  // FP32 op(A) and op(B)^T, rows contiguous: box of 32 rows x 64 K
  __nv_bfloat16* hi[2];
  __nv_bfloat16* lo[2];
  int* flags;          // one per chunk: A's (block * kb_stride + slab), then B's
  int* done;           // per block (A's, then B's): its chunks converted so far
  int* claim;          // the next chunk to convert
  int rows[2];         // M, N
  int blocks[2];       // ceil(rows / 128)
  int Kp, num_kb;
  int kb_stride;       // num_kb rounded up to 4: a block's flags, 16-byte aligned
  int pre[2];          // blocks [0, pre) of each operand: converted before the launch
  // a batch (the grouped leaf): the chunks in claim order, each (operand,
  // first row (a multiple of 128), first K element (of 64), flag index),
  // and the operands they name; flags and claim as above (the per-instance
  // flag bases are in the instances' records)
  const SplitTile* chunks;
  const SplitOp* ops;
  int num_chunks;
};

// ---- PTX helpers -----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// CLUSTER: acquire at cluster scope, for barriers that threads of the peer
// CTA of a pair arrive on.
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  if constexpr (CLUSTER) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  }
  return ok != 0;
}
__device__ __forceinline__ void st_cluster_u32(uint32_t cluster_addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}
// try_wait with a suspend-time hint: a thread whose phase is not complete
// sleeps at most about hint_ns (it wakes as soon as the phase completes), so
// a bounded wait regains control at a rate set by its own limit.
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  if constexpr (CLUSTER) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
  }
  return ok != 0;
}
// The hint of a bounded wait's polls: a quarter of its limit (the clock is
// read every fourth poll), at most 20 us, so a raised abort flag is seen
// within about 80 us even under the default 2 s limit.
__device__ __forceinline__ uint32_t poll_hint(uint64_t limit_ns) {
  const uint64_t h = limit_ns >> 2;
  return h < 32ull ? 32u : h > 20000ull ? 20000u : (uint32_t)h;
}
// Wait for the phase of `bar` with the given parity. Gives up (returns
// false) when another role raised the abort flag or after limit_ns, in
// which case it records `code` in the status word and raises the flag.
// peer_abort: shared::cluster address of the peer CTA's abort flag (a pair
// of CTAs on one tile), raised too so the peer stops waiting; 0 for none.
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int* status, int code, uint64_t limit_ns = WAIT_LIMIT_NS,
                                          uint32_t peer_abort = 0) {
  const uint32_t hint = poll_hint(limit_ns);
  if (mbar_try_wait_hint<CLUSTER>(bar, parity, hint)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t n = 1;; ++n) {
    if (mbar_try_wait_hint<CLUSTER>(bar, parity, hint)) return true;
    if ((n & 3u) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > limit_ns) {
        if (status) atomicOr_system(status, code);
        *abort_flag = 1;
        if (peer_abort) st_cluster_u32(peer_abort, 1);
        return false;
      }
    }
  }
}
// The same bounded wait for a whole warp, with one outcome for every lane:
// all lanes poll the barrier, and lane 0 alone decides to give up (abort
// raised, or the limit passed), so the warp never splits between the two
// outcomes.
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                               int* status, int code, uint64_t limit_ns = WAIT_LIMIT_NS,
                                               uint32_t peer_abort = 0) {
  const int lane = threadIdx.x & 31;
  const uint64_t t0 = globaltimer();
  const uint32_t hint = poll_hint(limit_ns);
  for (uint32_t n = 1;; ++n) {
    if (__all_sync(0xffffffffu, mbar_try_wait_hint<CLUSTER>(bar, parity, hint))) return true;
    if ((n & 3u) == 0) {
      int give_up = 0;
      if (lane == 0) {
        if (*abort_flag) {
          give_up = 1;
        } else if (globaltimer() - t0 > limit_ns) {
          if (status) atomicOr_system(status, code);
          *abort_flag = 1;
          if (peer_abort) st_cluster_u32(peer_abort, 1);
          give_up = 1;
        }
      }
      if (__shfl_sync(0xffffffffu, give_up, 0)) return false;
    }
  }
}
__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t cluster_addr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(cluster_addr) : "memory");
  return v;
}
// Count tx bytes as arrived on an mbarrier's current phase (the drain uses
// it for loads a stage expected that were never issued).
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int c0,
                                            int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
// The same load for one CTA of a pair (.cta_group::2): the mbarrier may be
// the peer's (a shared::cluster address), so both CTAs' loads of a stage
// complete on the leader CTA's barrier.
__device__ __forceinline__ void tma_load_2d_pair(const CUtensorMap* map, uint32_t bar_cluster, void* dst, int c0,
                                                 int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of the object at shared address a in CTA `rank`
__device__ __forceinline__ uint32_t mapa_rank(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// Every thread of both CTAs of the cluster (reachable from divergent code).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// Arrive on an mbarrier of either CTA of the pair (a shared::cluster
// address). The epilogue releases a tensor-memory buffer with it: its reads
// are complete (tcgen05.wait::ld) and ordered before the arrive by
// tcgen05.fence::before_thread_sync, so the arrive needs only the default
// CTA-scope release; a cluster-scope release stalled the epilogue warps on
// a memory barrier at every chunk (the BF16x3 leaf is 1% faster without it).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of tcgen05 (K-major, 64- or 128-byte
// swizzle): start address >> 4 in bits 0-13, leading byte offset >> 4 in
// 16-29 (not used by swizzled K-major layouts), stride byte offset >> 4 in
// 32-45 (the distance between groups of 8 rows: 8 * ROW_BYTES), descriptor
// version 1 in bits 46-47, swizzle mode in bits 61-63 (4 = 64-byte, 2 =
// 128-byte swizzle).
template <int ROW_BYTES>
__device__ __forceinline__ uint64_t sdesc_k(uint32_t saddr) {
  static_assert(ROW_BYTES == 64 || ROW_BYTES == 128, "64- or 128-byte swizzle");
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>((8 * ROW_BYTES) >> 4) << 32;      // 8-row group stride
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(ROW_BYTES == 128 ? 2 : 4) << 61;  // 128B / 64B swizzle
  return d;
}
// The same descriptor in two halves: the low word (address >> 4 in bits
// 0-13, shared-memory addresses below 256 KB, and the leading offset) varies
// with the address; the high word is a constant of the swizzle.
__device__ __forceinline__ uint32_t sdesc_lo(uint32_t saddr) { return ((saddr & 0x3FFFFu) >> 4) | (1u << 16); }
template <int ROW_BYTES>
__device__ __forceinline__ uint64_t sdesc_of(uint32_t lo) {
  return static_cast<uint64_t>(lo) | (sdesc_k<ROW_BYTES>(0) & 0xFFFFFFFF00000000ull);
}
// Instruction descriptor of tcgen05.mma kind::f16: D format F32 (bits 4-5 =
// 1), A and B BF16 (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}
// CG: 1 = this CTA's tensor core; 2 = the pair's (issued by the leader CTA:
// A's 256 rows are 128 in each CTA's shared memory, B's N rows N/2 in each,
// at the same offsets; D's rows 0-127 land in the leader's tensor memory and
// rows 128-255 in the peer's)
template <int CG>
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  if constexpr (CG == 2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}
// Instruction descriptor of tcgen05.mma kind::f8f6f4 with E4M3 A and B
// (format 0 in bits 7-9 and 10-12), F32 D, K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc_e4m3(int m, int n) {
  return (1u << 4) | (static_cast<uint32_t>(n >> 3) << 17) | (static_cast<uint32_t>(m >> 4) << 24);
}
template <int CG>
__device__ __forceinline__ void umma_e4m3(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  if constexpr (CG == 2) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}
// Arrive on `bar` once every MMA issued before has completed; CG 2 arrives on
// the barrier at the same offset in both CTAs of the pair.
template <int CG>
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  if constexpr (CG == 2) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
  } else {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
  }
}
// (a0, a1) <- (s*v0 + a0, s*v1 + a1), one rounding each (packed FP32 FMA).
__device__ __forceinline__ void ffma2(float& a0, float& a1, float s, uint32_t v0, uint32_t v1) {
  asm("{\n\t.reg .b64 acc, val, sc;\n\t"
      "mov.b64 acc, {%0, %1};\n\t"
      "mov.b64 val, {%3, %4};\n\t"
      "mov.b64 sc, {%2, %2};\n\t"
      "fma.rn.f32x2 acc, sc, val, acc;\n\t"
      "mov.b64 {%0, %1}, acc;\n\t}"
      : "+f"(a0), "+f"(a1)
      : "f"(s), "r"(v0), "r"(v1));
}
__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// All THREADS threads of the CTA, arriving from different branches: a
// named barrier without .aligned, which may be reached from divergent code.
__device__ __forceinline__ void cta_barrier_all() {
  asm volatile("barrier.sync 1, %0;" ::"n"(THREADS) : "memory");
}

// A 32-column tensor-memory load without its wait (several go in flight),
// and the wait that ends them; the wait takes the loaded registers as
// operands so nothing that reads them can be scheduled before it.
__device__ __forceinline__ void tmem_ld_x32_issue(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld_into(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                 "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                 "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]),
                 "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]),
                 "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

// Two 32-column tensor-memory loads in flight before one wait.
__device__ __forceinline__ void tmem_ld_2x32(uint32_t taddr0, uint32_t taddr1, uint32_t (&r)[32],
                                             uint32_t (&s)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr0));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]),
        "=r"(s[8]), "=r"(s[9]), "=r"(s[10]), "=r"(s[11]), "=r"(s[12]), "=r"(s[13]), "=r"(s[14]),
        "=r"(s[15]), "=r"(s[16]), "=r"(s[17]), "=r"(s[18]), "=r"(s[19]), "=r"(s[20]), "=r"(s[21]),
        "=r"(s[22]), "=r"(s[23]), "=r"(s[24]), "=r"(s[25]), "=r"(s[26]), "=r"(s[27]), "=r"(s[28]),
        "=r"(s[29]), "=r"(s[30]), "=r"(s[31])
      : "r"(taddr1));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---- operand split ------------------------------------------------------------
__device__ __forceinline__ void split_pair(float x, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  l = __float2bfloat16_rn(x - __bfloat162float(h));
}
// Three parts: x - hi is exact in FP32 (at most 16 significant bits), and so
// is (x - hi) - mid (at most 8), which lo then holds exactly.
__device__ __forceinline__ void split_three(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  const float r = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r);
  l = __float2bfloat16_rn(r - __bfloat162float(m));
}
// NPROD: 1 = hi only, 3 = hi and lo, 6 = hi, mid (in lo) and lo (in lo2)
template <int NPROD>
__device__ __forceinline__ void split_elem(float x, __nv_bfloat16& h, __nv_bfloat16& l, __nv_bfloat16& l2) {
  if constexpr (NPROD == 6) split_three(x, h, l, l2);
  else split_pair(x, h, l);
}

// X "m-major": element (r, k) at X[r + k*ld] (rows contiguous). One TR x TK
// tile (rows r0.., K k0..) per CTA of 256 threads, transposed through
// shared memory so both the FP32 read (TR rows of a column in a row) and
// the BF16 writes (TK elements of a plane row in a row) are coalesced.
template <int NPROD, int TR = 64, int TK = 64>
__device__ __forceinline__ void split_tile_m(const float* __restrict__ X, int64_t ld, int rows, int K, int Kp,
                                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                             __nv_bfloat16* __restrict__ lo2, int64_t r0, int64_t k0) {
  static_assert(TR % 32 == 0 && TK % 8 == 0 && (TR * TK) % 2048 == 0, "tile of whole warps and 8-K groups");
  constexpr int LOADS = TR * TK / 256, GROUPS = TR * TK / 8 / 256;
  __shared__ float t[TK][TR + 1];
  const int tid = threadIdx.x;
  // all loads of a thread in flight before the first shared-memory store
  float v[LOADS];
#pragma unroll
  for (int it = 0; it < LOADS; ++it) {
    const int e = tid + it * 256;
    const int kk = e / TR, rr = e % TR;
    const int64_t gr = r0 + rr, gk = k0 + kk;
    v[it] = (gr < rows && gk < K) ? __ldcs(X + gr + gk * ld) : 0.f;
  }
#pragma unroll
  for (int it = 0; it < LOADS; ++it) {
    const int e = tid + it * 256;
    t[e / TR][e % TR] = v[it];
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < GROUPS; ++it) {
    int e = tid + it * 256;
    int rr = e / (TK / 8), kc = (e % (TK / 8)) * 8;
    int64_t gr = r0 + rr, gk = k0 + kc;
    if (gr >= rows || gk >= Kp) continue;
    __align__(16) __nv_bfloat16 h[8];
    __align__(16) __nv_bfloat16 l[8];
    __align__(16) __nv_bfloat16 l2[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) split_elem<NPROD>(t[kc + u][rr], h[u], l[u], l2[u]);
    *reinterpret_cast<uint4*>(hi + gr * Kp + gk) = *reinterpret_cast<const uint4*>(h);
    if (NPROD >= 3) *reinterpret_cast<uint4*>(lo + gr * Kp + gk) = *reinterpret_cast<const uint4*>(l);
    if (NPROD == 6) *reinterpret_cast<uint4*>(lo2 + gr * Kp + gk) = *reinterpret_cast<const uint4*>(l2);
  }
}

// X "k-major": element (r, k) at X[k + r*ld] (K contiguous); one 64 x 64
// tile per CTA, eight consecutive K elements per thread and pass.
template <int NPROD>
__device__ __forceinline__ void split_tile_k(const float* __restrict__ X, int64_t ld, int rows, int K, int Kp,
                                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                             __nv_bfloat16* __restrict__ lo2, int64_t r0, int64_t k0) {
  // both passes' 16 loads in flight before the first conversion
  float v[2][8];
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int e = threadIdx.x + it * 256;
    const int64_t r = r0 + (e >> 3), k = k0 + (e & 7) * 8;
    const bool in = r < rows;
#pragma unroll
    for (int u = 0; u < 8; ++u) v[it][u] = (in && k + u < K) ? __ldcs(X + r * ld + k + u) : 0.f;
  }
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int e = threadIdx.x + it * 256;
    const int64_t r = r0 + (e >> 3), k = k0 + (e & 7) * 8;
    if (r >= rows || k >= Kp) continue;
    __align__(16) __nv_bfloat16 h[8];
    __align__(16) __nv_bfloat16 l[8];
    __align__(16) __nv_bfloat16 l2[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) split_elem<NPROD>(v[it][u], h[u], l[u], l2[u]);
    *reinterpret_cast<uint4*>(hi + r * Kp + k) = *reinterpret_cast<const uint4*>(h);
    if (NPROD >= 3) *reinterpret_cast<uint4*>(lo + r * Kp + k) = *reinterpret_cast<const uint4*>(l);
    if (NPROD == 6) *reinterpret_cast<uint4*>(lo2 + r * Kp + k) = *reinterpret_cast<const uint4*>(l2);
  }
}

// The tile of the single-operand split (the batch's pre-pass keeps 64 x 64).
// Long reads along the contiguous rows pay more than long plane-row writes
// (the K-adjacent tile's CTA runs soon after and completes the 32-byte
// sectors in L2): at M = N = K = 8192 the two splits of a step took 210 us
// with 64 x 64 tiles, 220-232 us with 128 x 64, 64 x 128 or 512 x 16,
// 208-213 us with 256 x 16 or 128 x 32, and 197-202 us with 256 x 32.
constexpr int SPLIT_TR = 256, SPLIT_TK = 32;
template <int NPROD>
__global__ void __launch_bounds__(256) split_mmajor(const float* __restrict__ X, int64_t ld, int rows, int K,
                                                    int Kp, __nv_bfloat16* __restrict__ hi,
                                                    __nv_bfloat16* __restrict__ lo, __nv_bfloat16* __restrict__ lo2) {
  split_tile_m<NPROD, SPLIT_TR, SPLIT_TK>(X, ld, rows, K, Kp, hi, lo, lo2, (int64_t)blockIdx.x * SPLIT_TR,
                                          (int64_t)blockIdx.y * SPLIT_TK);
}

// One operand of a batch and its planes; one 64 x 64 tile of one operand.
struct SplitOp {
  const float* X;
  int64_t ld;
  int mmajor, rows, K, Kp;
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
};
// A tile of the batch's split (64 x 64), or a chunk of its in-leaf
// conversion (128 rows x 64 K); flag: the in-leaf conversion's flag of its
// chunk, or -1.
struct SplitTile {
  int op, r0, k0, flag;
};

// The pre-pass of a whole batch in one launch: CTA i splits tile i. With
// in-leaf conversion (flags given) it splits only the chunks the leaf's
// first round reads and marks their flags; the leaf starts after this
// kernel has finished, so nothing more orders them.
template <int NPROD>
__global__ void __launch_bounds__(256) split_batch(const SplitOp* __restrict__ ops,
                                                   const SplitTile* __restrict__ tiles, int* flags) {
  const SplitTile t = tiles[blockIdx.x];
  const SplitOp o = ops[t.op];
  if (o.mmajor) split_tile_m<NPROD>(o.X, o.ld, o.rows, o.K, o.Kp, o.hi, o.lo, nullptr, t.r0, t.k0);
  else split_tile_k<NPROD>(o.X, o.ld, o.rows, o.K, o.Kp, o.hi, o.lo, nullptr, t.r0, t.k0);
  if (flags && t.flag >= 0 && threadIdx.x == 0) flags[t.flag] = 1;
}

// X "k-major": element (r, k) at X[k + r*ld] (K contiguous).
template <int NPROD>
__global__ void __launch_bounds__(256) split_kmajor(const float* __restrict__ X, int64_t ld, int rows, int K,
                                                    int Kp, __nv_bfloat16* __restrict__ hi,
                                                    __nv_bfloat16* __restrict__ lo, __nv_bfloat16* __restrict__ lo2) {
  const int64_t chunks = Kp / 8;
  const int64_t total = (int64_t)rows * chunks;
  for (int64_t task = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; task < total;
       task += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = task / chunks, k = (task % chunks) * 8;
    const float* src = X + r * ld + k;
    __align__(16) __nv_bfloat16 h[8];
    __align__(16) __nv_bfloat16 l[8];
    __align__(16) __nv_bfloat16 l2[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) split_elem<NPROD>((k + u < K) ? src[u] : 0.f, h[u], l[u], l2[u]);
    *reinterpret_cast<uint4*>(hi + r * Kp + k) = *reinterpret_cast<const uint4*>(h);
    if (NPROD >= 3) *reinterpret_cast<uint4*>(lo + r * Kp + k) = *reinterpret_cast<const uint4*>(l);
    if (NPROD == 6) *reinterpret_cast<uint4*>(lo2 + r * Kp + k) = *reinterpret_cast<const uint4*>(l2);
  }
}

// Y (rows x K; element (r, k) at X[k + r*ld] when KCONTIG, else X[r + k*ld])
// -> E4M3 codes q[r*Kp + k] and one FP32 scale per 128 x 128 block,
// scales[rb*nkb + kb] = amax / 448 (1 when the block is all zero), codes
// e4m3_rn_satfinite(x / scale). One CTA of 512 threads per block: thread t
// holds row t % 128, K elements 32 * (t / 128) .. + 31 of the block in
// registers (m-major source: each of its 32 loads reads 32 consecutive rows
// of one K column across the warp; K-contiguous: 8 float4 of its row). The
// block's amax comes from a warp shuffle and 16 partials in shared memory;
// each thread then quantises its 32 values (x / scale rounded as IEEE
// division rounds it) into a 128 x 128 byte tile, which the CTA writes out
// as 128-byte row segments.
constexpr int QTHREADS = 512;
constexpr int QROW = FP8_BLOCK + 16;  // byte tile row: 16-byte aligned, 144 B apart
template <bool KCONTIG, bool VEC>
__global__ void __launch_bounds__(QTHREADS, 2) quant_fp8(const float* __restrict__ X, int64_t ld, int rows, int K,
                                                         int Kp, uint8_t* __restrict__ q,
                                                         float* __restrict__ scales, int nkb) {
  __shared__ __align__(16) uint8_t codes[FP8_BLOCK * QROW];
  __shared__ float red[QTHREADS / 32];
  __shared__ float s_sh;
  const int tid = threadIdx.x;
  const int r = tid % FP8_BLOCK, kq = (tid / FP8_BLOCK) * 32;
  const int64_t r0 = (int64_t)blockIdx.x * FP8_BLOCK, k0 = (int64_t)blockIdx.y * FP8_BLOCK;
  const int64_t gr = r0 + r, gk = k0 + kq;
  const bool row_in = gr < rows;
  float v[32];
  if (KCONTIG) {
    const float* src = X + gk + gr * ld;
#pragma unroll
    for (int u = 0; u < 32; u += 4) {
      if (VEC && row_in && gk + u + 3 < K) {
        const float4 t = __ldcs(reinterpret_cast<const float4*>(src + u));
        v[u] = t.x, v[u + 1] = t.y, v[u + 2] = t.z, v[u + 3] = t.w;
      } else {
#pragma unroll
        for (int w = 0; w < 4; ++w) v[u + w] = (row_in && gk + u + w < K) ? __ldcs(src + u + w) : 0.f;
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < 32; ++u) v[u] = (row_in && gk + u < K) ? __ldcs(X + gr + (gk + u) * ld) : 0.f;
  }
  float amax = 0.f;
#pragma unroll
  for (int u = 0; u < 32; ++u) amax = fmaxf(amax, fabsf(v[u]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((tid & 31) == 0) red[tid >> 5] = amax;
  __syncthreads();
  if (tid == 0) {
    float m = red[0];
    for (int w = 1; w < QTHREADS / 32; ++w) m = fmaxf(m, red[w]);
    const float s = m > 0.f ? __fdiv_rn(m, 448.f) : 1.f;
    scales[(int64_t)blockIdx.x * nkb + blockIdx.y] = s;
    s_sh = s;
  }
  __syncthreads();
  const float s = s_sh;
  // x / s rounded to nearest, as IEEE division gives it. For s in
  // [2^-80, 2^80] (every block of real data) one correction step suffices
  // (Markstein's theorem: with rs = RN(1/s) and q0 = RN(x * rs) within an
  // ulp of x / s, the remainder e = x - q0 * s is exact in an FMA and
  // RN(q0 + e * rs) is the correctly rounded quotient; quotients that a
  // subnormal remainder could disturb are below 2^-10, which E4M3 rounds
  // to zero either way). Other scales take the IEEE division itself.
  const bool fast = s >= 0x1p-80f && s <= 0x1p80f;
  const float rs = __frcp_rn(s);
  auto quotient = [&](float x) {
    if (!fast) return __fdiv_rn(x, s);
    const float q0 = x * rs;
    return fmaf(fmaf(-q0, s, x), rs, q0);
  };
  // this thread's 32 codes, 4 to a word, into its row of the byte tile
  uint32_t w[8];
#pragma unroll
  for (int u = 0; u < 32; u += 4) {
    uint32_t b = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      b |= (uint32_t)__nv_cvt_float_to_fp8(quotient(v[u + e]), __NV_SATFINITE, __NV_E4M3) << (8 * e);
    w[u / 4] = b;
  }
  uint4* dst = reinterpret_cast<uint4*>(codes + r * QROW + kq);
  dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
  dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
  __syncthreads();
  // 128 rows x 8 segments of 16 bytes: a warp writes 4 rows of 128 bytes
  for (int i = tid; i < FP8_BLOCK * (FP8_BLOCK / 16); i += QTHREADS) {
    const int row = i / (FP8_BLOCK / 16), seg = (i % (FP8_BLOCK / 16)) * 16;
    const int64_t orow = r0 + row, ok = k0 + seg;
    if (orow >= rows || ok >= Kp) continue;
    *reinterpret_cast<uint4*>(q + orow * Kp + ok) = *reinterpret_cast<const uint4*>(codes + row * QROW + seg);
  }
}

// ---- the leaf kernel -------------------------------------------------------------
// Persistent: CTA b handles tiles b, b + gridDim.x, ... in a grouped order
// (GROUP_N column tiles at a time, N fastest within them) so CTAs that run
// together share operand panels in L2.
// Tail split of a persistent single-instance launch: when the last round of
// whole tiles would leave more than half of the units (CTAs or pairs) idle,
// each of its tiles runs as two K halves on two units. Returns how many
// tiles split (0: none). Host and kernel take the decision with this one
// function, from the same tile count, unit count and K slabs.
__host__ __device__ constexpr int tail_split_tiles(int tiles, int units, int num_kb) {
  return (units > 0 && tiles >= units && tiles % units > 0 && 2 * (tiles % units) <= units && num_kb >= 4)
             ? tiles % units
             : 0;
}

// The leaf variants built with the tail split: BF16 and BF16x3 on pairs,
// plain or with the tanh leaf merged (BF16 only). In the others (FP8, the
// tanh adjoint, BF16x3 with tanh) ptxas spilled more of the epilogue's
// registers with the split compiled in.
__host__ __device__ constexpr bool tail_split_variant(int mode, int epi, bool grouped) {
  return !grouped && mode != 8 && (epi == 0 || (epi == 1 && mode == 1));
}

__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int tile_rows, int tile_cols, int* m0,
                                            int* n0) {
  const int group = GROUP_N * tiles_m;
  const int g = t / group, r = t % group;
  const int first_n = g * GROUP_N;
  const int gn = min(GROUP_N, tiles_n - first_n);
  *m0 = (r / gn) * tile_rows;
  *n0 = (first_n + r % gn) * tile_cols;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// four consecutive flags (16-byte aligned) as a 4-bit mask of the nonzero ones
__device__ __forceinline__ uint32_t ld_relaxed_mask4(const int* p) {
  int a, b, c, d;
  asm volatile("ld.relaxed.gpu.global.v4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(a), "=r"(b), "=r"(c), "=r"(d)
               : "l"(p)
               : "memory");
  return (a != 0 ? 1u : 0u) | (b != 0 ? 2u : 0u) | (c != 0 ? 4u : 0u) | (d != 0 ? 8u : 0u);
}
// acquire for what relaxed loads observed, extended to the TMA (async
// proxy) loads that follow
__device__ __forceinline__ void fence_acquire_for_tma() {
  asm volatile("fence.acq_rel.gpu;\n\tfence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// Wait until *flag is nonzero (a chunk of planes written by a converter
// warp), bounded as mbar_wait is; then order the TMA loads that follow
// after the converter's writes.
__device__ __forceinline__ bool flag_wait(const int* flag, volatile int* abort_flag, int* status, int code,
                                          uint32_t peer_abort, uint64_t limit_ns) {
  if (ld_acquire_gpu(flag) == 0) {
    const uint64_t t0 = globaltimer();
    for (uint32_t n = 1;; ++n) {
      if (ld_acquire_gpu(flag) != 0) break;
      if ((n & 15u) == 0) {
        if (*abort_flag) return false;
        if (globaltimer() - t0 > limit_ns) {
          if (status) atomicOr_system(status, code);
          *abort_flag = 1;
          if (peer_abort) st_cluster_u32(peer_abort, 1);
          return false;
        }
      }
    }
  }
  asm volatile("fence.proxy.async.global;" ::: "memory");
  return true;
}

// One converter warp of the in-leaf conversion (see ConvParams). tab: the
// round table (R at [CV_MAX_ROUNDS * CV_TAB], round r's A blocks [lo, hi),
// B blocks [lo, hi) and first chunk at [r * CV_TAB ...], the chunk total at
// [R * CV_TAB + 4]); bar, buf: this warp's two piece barriers and staging
// buffers. Claims chunks until none is left or the kernel aborts.
__device__ __forceinline__ void cv_convert(const ConvParams& cv, const int* tab, uint64_t* bar, uint8_t* buf,
                                        int lane, volatile int* abort_flag, int* status, uint64_t limit_ns) {
  const int R = tab[CV_MAX_ROUNDS * CV_TAB];
  const int total = tab[R * CV_TAB + 4];
  int r = 0;  // round cursor (a warp's claims only increase)
  struct Piece {
    int op, blk, kb, j;
  };
  // claim a chunk (lane 0; the whole warp gets it) and place its first piece
  auto next_chunk = [&](Piece& q) -> bool {
    int c = total;
    if (lane == 0 && !*abort_flag) c = atomicAdd(cv.claim, 1);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c >= total) return false;
    while (r + 1 < R && c >= tab[(r + 1) * CV_TAB + 4]) ++r;
    const int* e = tab + r * CV_TAB;
    const int na = e[1] - e[0], n = na + (e[3] - e[2]);
    const int i = c - e[4];
    const int b = i % n;
    q.kb = i / n;
    q.op = b < na ? 0 : 1;
    q.blk = q.op ? e[2] + (b - na) : e[0] + b;
    q.j = 0;
    return true;
  };
  // TMA load of a piece (32 rows x 64 K of FP32) into buffer b; every
  // lane's reads of that buffer are complete (the caller syncs the warp)
  auto issue = [&](const Piece& q, int b) {
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bar[b], CV_PIECE_BYTES);
      tma_load_2d(&cv.src[q.op], &bar[b], buf + b * CV_PIECE_BYTES, q.blk * CV_ROWS + q.j * CV_PIECE,
                  q.kb * CV_BK);
    }
  };
  Piece cur, nxt;
  if (!next_chunk(cur)) return;
  issue(cur, 0);
  int b = 0;
  // per buffer (bit b): the parity of its next phase, and whether a load was
  // issued into it and not yet waited for
  uint32_t ph = 0u, inflight = 1u;
  for (;;) {
    bool has_next;
    if (cur.j + 1 < CV_PIECES) {
      nxt = cur;
      ++nxt.j;
      has_next = !*abort_flag;
    } else {
      has_next = next_chunk(nxt);
    }
    __syncwarp();  // the piece converted last (buffer b ^ 1) is read by every lane
    if (has_next) {
      issue(nxt, b ^ 1);
      inflight |= 1u << (b ^ 1);
    }
    if (!mbar_wait_warp(&bar[b], (ph >> b) & 1u, abort_flag, status, ST_CONVERT, limit_ns)) break;
    inflight &= ~(1u << b);
    ph ^= 1u << b;
    // The stage holds element (row i, k) at k * 32 + i. Lane l converts K
    // elements 8 (l % 8) .. + 7 of rows l / 8 + 4 t (t = 0..7), so each
    // store instruction writes four whole 128-byte plane rows (eight lanes a
    // row) instead of 32 partial ones; its shared-memory reads conflict
    // eight ways, which costs little next to the leaf's own traffic.
    const float* st = reinterpret_cast<const float*>(buf + b * CV_PIECE_BYTES);
    const int g8 = (lane & 7) * 8;
    const int k0 = cur.kb * CV_BK + g8;
    if (k0 < cv.Kp) {
      __nv_bfloat16* hp = cv.hi[cur.op] + k0;
      __nv_bfloat16* lp = cv.lo[cur.op] + k0;
#pragma unroll 1
      for (int t = 0; t < CV_PIECE / 4; ++t) {
        const int r = (lane >> 3) + 4 * t;
        const int row = cur.blk * CV_ROWS + cur.j * CV_PIECE + r;
        if (row < cv.rows[cur.op]) {
          __align__(16) __nv_bfloat16 h[8];
          __align__(16) __nv_bfloat16 l[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) split_pair(st[(g8 + u) * CV_PIECE + r], h[u], l[u]);
          *reinterpret_cast<uint4*>(hp + (int64_t)row * cv.Kp) = *reinterpret_cast<const uint4*>(h);
          *reinterpret_cast<uint4*>(lp + (int64_t)row * cv.Kp) = *reinterpret_cast<const uint4*>(l);
        }
      }
    }
    if (cur.j + 1 == CV_PIECES) {
      // the chunk's planes are written: make them visible to the TMA loads
      // of other CTAs, then release its flag
      asm volatile("fence.proxy.async.global;" ::: "memory");
      __threadfence();
      __syncwarp();
      if (lane == 0) {
        const int blk = (cur.op ? cv.blocks[0] : 0) + cur.blk;
        st_release_gpu(cv.flags + (int64_t)blk * cv.kb_stride + cur.kb, 1);
        asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(cv.done + blk) : "memory");
      }
    }
    if (!has_next) break;
    cur = nxt;
    b ^= 1;
  }
  // leaving early (an abort, or a piece that never arrived): wait (bounded)
  // for this warp's loads still in flight before the CTA may exit
  __syncwarp();
  if (lane == 0) {
    for (int bb = 0; bb < 2; ++bb) {
      if (!((inflight >> bb) & 1u)) continue;
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&bar[bb], (ph >> bb) & 1u)) {
        if (globaltimer() - t0 > WAIT_LIMIT_NS) {
          if (status) atomicOr_system(status, ST_DRAIN);
          break;
        }
      }
    }
  }
  __syncwarp();
}

// 4-byte asynchronous copy global -> shared (src_bytes 0: the destination is
// zero-filled and nothing is read).
__device__ __forceinline__ void cp_async4(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One converter warp of a batch's in-leaf conversion: the chunks of
// cv.chunks in claim order, each in four pieces of 32 rows x 64 K staged by
// 4-byte cp.async copies (any leading dimension, either layout of the FP32
// operand; zeros past its rows and K) into two buffers, the next piece in
// flight while this one is converted. A piece holds element (row i, k) at
// k * 32 + (i ^ k % 32), so both layouts' copies and the conversion's reads
// spread over the banks. The conversion and the release of the chunk's flag
// are cv_convert's. cp.async waits on the warp's own copies only, which
// always complete.
__device__ __forceinline__ void cv_convert_batch(const ConvParams& cv, uint8_t* buf, int lane,
                                                 volatile int* abort_flag) {
  auto claim = [&]() -> int {
    int c = cv.num_chunks;
    if (lane == 0 && !*abort_flag) c = atomicAdd(cv.claim, 1);
    return __shfl_sync(0xffffffffu, c, 0);
  };
  auto stage = [&](int c, int j, int b) {
    const SplitTile ch = cv.chunks[c];
    const SplitOp o = cv.ops[ch.op];
    float* st = reinterpret_cast<float*>(buf + b * CV_PIECE_BYTES);
    const int r0 = ch.r0 + j * CV_PIECE;
    if (o.mmajor) {
      // element (r, k) at X[r + k ld]: lane l copies row r0 + l of each K column
      const int r = r0 + lane;
#pragma unroll 4
      for (int k = 0; k < CV_BK; ++k) {
        const int kk = ch.k0 + k;
        const bool in = r < o.rows && kk < o.K;
        cp_async4(st + k * CV_PIECE + (lane ^ (k & 31)), in ? o.X + (int64_t)kk * o.ld + r : o.X, in ? 4u : 0u);
      }
    } else {
      // element (r, k) at X[k + r ld]: lane l copies K elements l and l + 32 of each row
#pragma unroll 4
      for (int i = 0; i < CV_PIECE; ++i) {
        const int r = r0 + i;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = lane + 32 * h, kk = ch.k0 + k;
          const bool in = r < o.rows && kk < o.K;
          cp_async4(st + k * CV_PIECE + (i ^ lane), in ? o.X + (int64_t)r * o.ld + kk : o.X, in ? 4u : 0u);
        }
      }
    }
    cp_async_commit();
  };
  int c = claim();
  if (c >= cv.num_chunks) return;
  stage(c, 0, 0);
  int j = 0, b = 0;
  for (;;) {
    // the next piece: of this chunk, or of the next claimed one
    int nc = c, nj = j + 1;
    if (nj == CV_PIECES) {
      nc = claim();
      nj = 0;
    }
    const bool has_next = nc < cv.num_chunks;
    __syncwarp();  // every lane is done reading buffer b ^ 1 (the piece converted last)
    if (has_next) {
      stage(nc, nj, b ^ 1);
      cp_async_wait<1>();  // this piece's copies (the next one's may still fly)
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();  // every lane's copies of this piece are visible to the warp
    const SplitTile ch = cv.chunks[c];
    const SplitOp o = cv.ops[ch.op];
    const float* st = reinterpret_cast<const float*>(buf + b * CV_PIECE_BYTES);
    const int g8 = (lane & 7) * 8;
    const int k0 = ch.k0 + g8;
    if (k0 < o.Kp) {
      __nv_bfloat16* hp = o.hi + k0;
      __nv_bfloat16* lp = o.lo + k0;
#pragma unroll 1
      for (int t = 0; t < CV_PIECE / 4; ++t) {
        const int r = (lane >> 3) + 4 * t;
        const int row = ch.r0 + j * CV_PIECE + r;
        if (row < o.rows) {
          __align__(16) __nv_bfloat16 h[8];
          __align__(16) __nv_bfloat16 l[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int k = g8 + u;
            split_pair(st[k * CV_PIECE + (r ^ (k & 31))], h[u], l[u]);
          }
          *reinterpret_cast<uint4*>(hp + (int64_t)row * o.Kp) = *reinterpret_cast<const uint4*>(h);
          *reinterpret_cast<uint4*>(lp + (int64_t)row * o.Kp) = *reinterpret_cast<const uint4*>(l);
        }
      }
    }
    if (j + 1 == CV_PIECES) {
      // the chunk's planes are written: visible to other CTAs' TMA loads,
      // then its flag released
      asm volatile("fence.proxy.async.global;" ::: "memory");
      __threadfence();
      __syncwarp();
      if (lane == 0) st_release_gpu(cv.flags + ch.flag, 1);
    }
    if (!has_next) break;
    c = nc;
    j = nj;
    b ^= 1;
  }
  cp_async_wait<0>();
  __syncwarp();
}

// One instance of a batch of independent sgemm DFGs (device memory): its
// four operand-plane tensor maps (64-byte aligned), its result, and the tile
// width bn (64, 128 or 256 columns) its schedule chose.
struct GroupInst {
  CUtensorMap tm[4];  // A hi, A lo, B hi, B lo
  float* C;
  int64_t ldc;
  int M, N, K, bn;
  float alpha, beta;
  // in-leaf conversion: the flags of A's 128-row blocks start at flag_a
  // (block b's slab k at flag_a + b kb_stride + k), B's at flag_b
  int flag_a, flag_b, kb_stride;
  int pad[7];
};
static_assert(sizeof(GroupInst) % 64 == 0, "tensor maps stay 64-byte aligned in an array");
// One output tile of the batch's schedule, with what every role needs of
// its instance besides the tensor maps: one 64-byte load per tile, issued a
// tile ahead.
struct GroupTile {
  int inst, m0, n0, K;
  int M, N, bn, pad0;
  float* C;
  int64_t ldc;
  float alpha, beta;
  int pad1[2];
};
static_assert(sizeof(GroupTile) == 64, "one 64-byte record per tile");
struct GroupParams {
  const GroupInst* insts;
  const GroupTile* tiles;
  int num_tiles;
};

// What one tile needs: its instance's operands and result, and where it sits.
struct TileView {
  const CUtensorMap* tm[4];  // A hi, A lo, B hi, B lo (BF16x6's third planes: the kernel's tmA_lo2, tmB_lo2)
  float* C;
  int64_t ldc;
  int M, N, K, bn, m0, n0;
  float alpha, beta;
  int kb0, kb1;  // the K slabs this unit accumulates
  int part;      // tail split: which K half (0, 1), else -1
  int tail;      // tail split: the tile's index among the split tiles
};

// EPI: 0 none; 1 C = tanh(alpha*acc + beta*C); 2 C = (alpha*acc + beta*C)*(1 - H^2)
// (the elementwise leaf merged into the sgemm leaf, MergeDependentNodes).
// GROUPED: the persistent CTAs (or pairs) walk the tile list of a batch of
// instances (gp) instead of the tiles of the one instance of the kernel
// parameters; a tile is BM (PAIR: 2 BM) rows by its instance's width bn.
// PAIR: launched in clusters of 2 CTAs; each cluster takes 256 x 256 tiles
// (256 x bn when GROUPED; the internal node's instance maps to a CTA pair)
// and the leader CTA (rank 0) issues the pair's MMAs. Roles per CTA:
//   warp 0      TMA producer (both CTAs: each loads its own half)
//   warp 1      tensor-memory allocation; MMA issuer (leader only)
//   warps 2, 3  idle (they complete the control warpgroup), or CONVERT
//   warps 4-11  epilogue (both CTAs: each drains its own 128 rows)
// CONVERT: warps 2 and 3 write the operand planes (see ConvParams; a batch
// (GROUPED): cv_convert_batch) and the producer waits for each slab's
// chunks.
template <int MODE, int EPI, bool GROUPED, bool PAIR, bool CONVERT = false>
__global__ void __launch_bounds__(THREADS, 1)
    sgemm_tc(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
             const __grid_constant__ CUtensorMap tmB_hi, const __grid_constant__ CUtensorMap tmB_lo,
             const __grid_constant__ CUtensorMap tmA_lo2, const __grid_constant__ CUtensorMap tmB_lo2,
             TcParams p, GroupParams gp, const __grid_constant__ ConvParams cv) {
  static_assert(!(GROUPED && PAIR) || (EPI == 0 && MODE != 8 && MODE != 6),
                "batches on pairs: the BF16x3 and BF16 leaves, plain epilogue");
  static_assert(!CONVERT || (MODE == 3 && PAIR && Cfg<MODE, PAIR>::BK == CV_BK),
                "in-leaf conversion: the BF16x3 leaf on pairs, one chunk per slab");
  static_assert(MODE != 6 || (!GROUPED && EPI == 0), "BF16x6: single instances, plain epilogue");
  using C_ = Cfg<MODE, PAIR>;
  constexpr int CG = PAIR ? 2 : 1;
  constexpr int TM = PAIR ? 2 * BM : BM;  // tile rows (one CTA, or the pair)
  constexpr int S = C_::STAGES;
  constexpr int NPROD = MODE == 3 ? 3 : MODE == 6 ? 6 : 1;
  constexpr int BK = C_::BK, MMA_K = C_::MMA_K, KC_SLABS = C_::KC_SLABS;
  if (PAIR && cluster_nctarank() != 2) {
    // launched without its cluster: nothing was set up yet, so just report
    if (threadIdx.x == 0 && p.status) atomicOr_system(p.status, ST_CONFIG);
    return;
  }
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * C_::STAGE_BYTES);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;      // [NBUF] MMA -> epilogue: chunk accumulated in buffer b
  uint64_t* tempty = tfull + C_::NBUF;  // [NBUF] epilogue -> MMA: buffer b read out
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + C_::NBUF);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  // CONVERT: two piece barriers per converter warp (in the barrier area),
  // their staging buffers and the chunk order's round table after it
  uint64_t* cvbar = reinterpret_cast<uint64_t*>(smem + S * C_::STAGE_BYTES + 256);
  // the drain's barrier (a last MMA commit arrives on it) and the stages
  // this CTA's producer issued, read by the leader of a pair when it drains
  uint64_t* drainbar = reinterpret_cast<uint64_t*>(smem + S * C_::STAGE_BYTES + 288);
  volatile int* issued_sh = reinterpret_cast<volatile int*>(smem + S * C_::STAGE_BYTES + 296);
  // GROUPED pairs: the bytes this CTA's producer loaded into each stage (a
  // batch's tiles differ in width), for the drain's reconciliation
  uint32_t* stage_bytes_sh = reinterpret_cast<uint32_t*>(smem + S * C_::STAGE_BYTES + 304);
  static_assert(304 + 4 * C_::STAGES <= 512, "stage byte counts inside the barrier area");
  static_assert(2 * C_::STAGES * 8 + 2 * C_::NBUF * 8 + 8 <= 256, "barriers before the converters' and the drain's");
  const uint64_t limit_ns = wait_limit(p);
  uint8_t* cvbuf = smem + S * C_::STAGE_BYTES + 512;
  int* cvtab = reinterpret_cast<int*>(cvbuf + CV_WARPS * 2 * CV_PIECE_BYTES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;  // CTA within the pair
  const bool leader = rank == 0;
  const int unit = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;  // CTA or pair index
  const int num_units = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  // the peer's abort flag (raised with ours, so it stops waiting for us)
  const uint32_t peer_abort = PAIR ? mapa_rank(smem_u32((const void*)abort_flag), rank ^ 1u) : 0u;
  constexpr int TN = C_::TN, NBUF = C_::NBUF;
  const int tiles_m = (p.M + TM - 1) / TM, tiles_n = (p.N + TN - 1) / TN;
  const int num_tiles = GROUPED ? gp.num_tiles : tiles_m * tiles_n;
  // Work units: the tiles, except that a tail split (split_ws given) runs
  // each of the last n_split tiles as two units, one per K half. Both
  // halves write their partial sums to split_ws; the second to arrive adds
  // the other's and writes C (a + b == b + a: the same C whichever is
  // second), the first is done with the tile.
  // (compiled in where it leaves ptxas's register allocation as it was)
  constexpr bool TAIL = tail_split_variant(MODE, EPI, GROUPED);
  const int num_kb_all = GROUPED ? 0 : (p.K + BK - 1) / BK;
  const int n_split = (TAIL && p.split_ws) ? tail_split_tiles(num_tiles, num_units, num_kb_all) : 0;
  const int split_base = num_tiles - n_split;
  const int num_work = num_tiles + n_split;
  auto work_tile = [&](int t, int* part) {
    *part = -1;
    if (t < split_base) return t;
    *part = (t - split_base) & 1;
    return split_base + ((t - split_base) >> 1);
  };

  // GROUPED: tile t's record (an empty one past the end); the roles load the
  // next tile's record while they work on the current one
  auto fetch = [&](int t) {
    GroupTile gt{};
    if constexpr (GROUPED) {
      if (t < num_tiles) gt = gp.tiles[t];
    }
    return gt;
  };
  auto view = [&](int t, const GroupTile& gt) {
    TileView v;
    if constexpr (GROUPED) {
      const GroupInst* in = gp.insts + gt.inst;
      for (int i = 0; i < 4; ++i) v.tm[i] = &in->tm[i];
      v.C = gt.C;
      v.ldc = gt.ldc;
      v.M = gt.M;
      v.N = gt.N;
      v.K = gt.K;
      v.bn = gt.bn;
      v.alpha = gt.alpha;
      v.beta = gt.beta;
      v.m0 = gt.m0;
      v.n0 = gt.n0;
      v.kb0 = 0;
      v.kb1 = (gt.K + BK - 1) / BK;
      v.part = -1;
      v.tail = 0;
    } else {
      v.tm[0] = &tmA_hi;
      v.tm[1] = &tmA_lo;
      v.tm[2] = &tmB_hi;
      v.tm[3] = &tmB_lo;
      v.C = p.C;
      v.ldc = p.ldc;
      v.M = p.M;
      v.N = p.N;
      v.K = p.K;
      v.bn = TN;
      v.alpha = p.alpha;
      v.beta = p.beta;
      if constexpr (TAIL) {
        const int tile = work_tile(t, &v.part);
        tile_coords(tile, tiles_m, tiles_n, TM, TN, &v.m0, &v.n0);
        v.kb0 = v.part == 1 ? num_kb_all / 2 : 0;
        v.kb1 = v.part == 0 ? num_kb_all / 2 : num_kb_all;
        v.tail = tile - split_base;
      } else {
        tile_coords(t, tiles_m, tiles_n, TM, TN, &v.m0, &v.n0);
        v.kb0 = 0;
        v.kb1 = num_kb_all;
        v.part = -1;
        v.tail = 0;
      }
    }
    return v;
  };

  // stage s: the PLANES planes of A, then those of B ([A hi][A lo][A lo2]
  // [B hi][B lo][B lo2]; lo planes for NPROD 3 and 6, lo2 for 6)
  auto a_pl = [&](int s, int i) { return smem + s * C_::STAGE_BYTES + i * C_::A_SLAB; };
  auto b_pl = [&](int s, int i) { return smem + s * C_::STAGE_BYTES + C_::PLANES * C_::A_SLAB + i * C_::B_SLAB; };
  auto a_hi = [&](int s) { return a_pl(s, 0); };
  auto b_hi = [&](int s) { return b_pl(s, 0); };

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], PAIR ? 2 * EPI_WARPS : EPI_WARPS);  // PAIR: both CTAs' epilogues
    }
    *abort_flag = 0;
    mbar_init(drainbar, 1);
    *issued_sh = 0;
    if constexpr (CONVERT && !GROUPED) {
      for (int b = 0; b < 2 * CV_WARPS; ++b) mbar_init(&cvbar[b], 1);
      // Round r of the grouped order runs tiles [r U, (r + 1) U) (U units).
      // Row tile rt is first used by tile rt * gn0 (group 0), column tile
      // ct by tile (ct / GROUP_N) * GROUP_N * tiles_m + ct % GROUP_N: round
      // r converts the 128-row blocks of the row and column tiles first used
      // in it (the last round: all the rest).
      const int U = num_units;
      const int gn0 = min(GROUP_N, tiles_n);
      const int R = max(1, min(CV_MAX_ROUNDS, (num_tiles + U - 1) / U));
      int ct = 0, base = 0;
      for (int r = 0; r < R; ++r) {
        const bool last = r + 1 == R;
        const int rt_lo = min(tiles_m, (r * U + gn0 - 1) / gn0);
        const int rt_hi = last ? tiles_m : min(tiles_m, ((r + 1) * U + gn0 - 1) / gn0);
        const int ct_lo = ct;
        while (ct < tiles_n && (last || (ct / GROUP_N) * GROUP_N * tiles_m + ct % GROUP_N < (r + 1) * U)) ++ct;
        int* e = cvtab + r * CV_TAB;
        e[1] = min(cv.blocks[0], 2 * rt_hi);
        e[0] = min(e[1], max(cv.pre[0], 2 * rt_lo));
        e[3] = min(cv.blocks[1], 2 * ct);
        e[2] = min(e[3], max(cv.pre[1], 2 * ct_lo));
        e[4] = base;
        base += ((e[1] - e[0]) + (e[3] - e[2])) * cv.num_kb;
      }
      cvtab[R * CV_TAB + 4] = base;  // the total: every chunk once
      cvtab[CV_MAX_ROUNDS * CV_TAB] = R;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    // PAIR: one warp of each CTA of the pair allocates, collectively
    if constexpr (PAIR) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  if constexpr (PAIR)
    cluster_sync_all();  // both CTAs' barriers exist before either signals the other's
  else
    __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // bookkeeping for the drain after an abort
  int issued = 0;     // producer: slabs requested (ring position)

  if (warp < EPI_WARP0) {
    // control warpgroup: its registers go to the epilogue warpgroups
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(RegSplit<MODE, EPI, PAIR, CONVERT>::CTRL_R));
    if (warp == 0 && lane == 0) {
      // ---- producer: TMA loads of the operand slabs into the ring. PAIR:
      // this CTA's 128 rows of A and its half of B's rows; both CTAs' loads
      // complete on the leader's barrier, which expects the pair's bytes.
      if (!GROUPED) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA_hi)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB_hi)) : "memory");
      }
      int it = 0;
      bool go = true;
      GroupTile nx = fetch(unit);
      for (int t = unit; go && t < num_work; t += num_units) {
        const GroupTile cur = nx;
        nx = fetch(t + num_units);
        const TileView v = view(t, cur);
        // this CTA's rows of B: PAIR, half of the tile's (B_ROWS, or bn / 2 of
        // a batch's tile of width bn); single CTAs all bn
        const int b_half = PAIR ? (GROUPED ? v.bn / 2 : C_::B_ROWS) : 0;
        const uint32_t b_rows = PAIR ? (uint32_t)b_half : (uint32_t)v.bn;
        const uint32_t bytes = C_::PLANES * (C_::A_SLAB + b_rows * C_::ROW_BYTES);
        const int ma = v.m0 + (int)rank * BM;
        const int nb = v.n0 + (int)rank * b_half;
        const int kb_hi = TAIL ? v.kb1 : (v.K + BK - 1) / BK;
        // CONVERT: whether every chunk of this CTA's A block, and of its B
        // block, is ready (split before the launch, or all converted): such
        // an operand needs no flag checks in this tile; for the other, the
        // flags of slabs [grp, grp + 4) seen set (bit per slab)
        bool done_a = true, done_b = true;
        int grp = -4;
        uint32_t ready_a = 0xFu, ready_b = 0xFu;
        const int* flag_a = nullptr;
        const int* flag_b = nullptr;
        if constexpr (CONVERT && GROUPED) {
          // a batch: this CTA's A block and B block (its bn / 2 rows of B lie
          // in one 128-row block) of the tile's instance; a block split
          // before the launch has its flags set
          const GroupInst* in = gp.insts + cur.inst;
          flag_a = cv.flags + in->flag_a + (int64_t)(ma / CV_ROWS) * in->kb_stride;
          flag_b = cv.flags + in->flag_b + (int64_t)(nb / CV_ROWS) * in->kb_stride;
          done_a = ma >= v.M;
          done_b = nb >= v.N;
          if (done_a && done_b) fence_acquire_for_tma();
        } else if constexpr (CONVERT) {
          const int ba = ma / CV_ROWS, bb = cv.blocks[0] + nb / CV_ROWS;
          flag_a = cv.flags + (int64_t)ba * cv.kb_stride;
          flag_b = cv.flags + (int64_t)bb * cv.kb_stride;
          done_a = ma >= p.M || ba < cv.pre[0] || ld_relaxed_gpu(cv.done + ba) == cv.num_kb;
          done_b = nb >= p.N || nb / CV_ROWS < cv.pre[1] || ld_relaxed_gpu(cv.done + bb) == cv.num_kb;
          if (done_a && done_b) fence_acquire_for_tma();
        }
        for (int kb = TAIL ? v.kb0 : 0; kb < kb_hi; ++kb, ++it) {
          const int s = it % S;
          const uint32_t ph = (it / S) & 1;
          if (!mbar_wait<PAIR>(&empty[s], ph ^ 1, abort_flag, p.status, ST_PRODUCER, limit_ns, peer_abort)) {
            go = false;
            break;
          }
          const int k = kb * BK;
          if constexpr (CONVERT) {
            // the chunks of this CTA's A rows and B rows for slab kb
            if (!(done_a && done_b)) {
              if ((kb & ~3) != grp) {
                grp = kb & ~3;
                ready_a = done_a ? 0xFu : ld_relaxed_mask4(flag_a + grp);
                ready_b = done_b ? 0xFu : ld_relaxed_mask4(flag_b + grp);
              }
              const uint32_t bit = 1u << (kb & 3);
              if (((ready_a & bit) == 0 &&
                   !flag_wait(flag_a + kb, abort_flag, p.status, ST_PRODUCER | ST_CONVERT, peer_abort, limit_ns)) ||
                  ((ready_b & bit) == 0 &&
                   !flag_wait(flag_b + kb, abort_flag, p.status, ST_PRODUCER | ST_CONVERT, peer_abort, limit_ns))) {
                go = false;
                break;
              }
              ready_a |= bit;
              ready_b |= bit;
              fence_acquire_for_tma();
            }
          }
          if constexpr (PAIR) {
            if constexpr (GROUPED) stage_bytes_sh[s] = bytes;
            if (leader) mbar_expect_tx(&full[s], 2 * bytes);
            const uint32_t bar = mapa_rank(smem_u32(&full[s]), 0);
            tma_load_2d_pair(v.tm[0], bar, a_hi(s), k, ma);
            if (NPROD >= 3) tma_load_2d_pair(v.tm[1], bar, a_pl(s, 1), k, ma);
            if constexpr (NPROD == 6) tma_load_2d_pair(&tmA_lo2, bar, a_pl(s, 2), k, ma);
            tma_load_2d_pair(v.tm[2], bar, b_hi(s), k, nb);
            if (NPROD >= 3) tma_load_2d_pair(v.tm[3], bar, b_pl(s, 1), k, nb);
            if constexpr (NPROD == 6) tma_load_2d_pair(&tmB_lo2, bar, b_pl(s, 2), k, nb);
          } else {
            mbar_expect_tx(&full[s], bytes);
            tma_load_2d(v.tm[0], &full[s], a_hi(s), k, ma);
            if (NPROD >= 3) tma_load_2d(v.tm[1], &full[s], a_pl(s, 1), k, ma);
            if constexpr (NPROD == 6) tma_load_2d(&tmA_lo2, &full[s], a_pl(s, 2), k, ma);
            tma_load_2d(v.tm[2], &full[s], b_hi(s), k, nb);
            if (NPROD >= 3) tma_load_2d(v.tm[3], &full[s], b_pl(s, 1), k, nb);
            if constexpr (NPROD == 6) tma_load_2d(&tmB_lo2, &full[s], b_pl(s, 2), k, nb);
          }
          issued = it + 1;
        }
        if (GROUPED && t + num_units < num_tiles && nx.K > 0) {
          // the next tile's instance: its tensor maps into the TMA unit's cache
          // (an instance with K = 0 has none)
          const GroupInst* in = gp.insts + nx.inst;
          for (int i = 0; i < (NPROD == 3 ? 4 : 3); i += (NPROD == 3 ? 1 : 2))
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&in->tm[i])) : "memory");
        }
      }
      *issued_sh = issued;  // for the drain (read by the pair's leader)
    } else if (warp == 1 && lane == 0 && leader) {
      // ---- MMA issuer: per K chunk, a fresh accumulation in tensor-memory
      // buffer (chunk parity); three (or one) products per K step
      int it = 0, g = 0;
      bool go = true;
      GroupTile nx = fetch(unit);
      for (int t = unit; go && t < num_work; t += num_units) {
        const GroupTile cur = nx;
        nx = fetch(t + num_units);
        const TileView v = view(t, cur);
        const int kb_lo = TAIL ? v.kb0 : 0, kb_hi = TAIL ? v.kb1 : (v.K + BK - 1) / BK;
        const int num_chunks = (kb_hi - kb_lo + KC_SLABS - 1) / KC_SLABS;
        const int n_mma = GROUPED ? v.bn : TN;
        const uint32_t idesc = C_::FP8 ? idesc_e4m3(TM, n_mma) : idesc_bf16(TM, n_mma);
        for (int c = 0; go && c < num_chunks; ++c, ++g) {
          const int buf = g % NBUF;
          const uint32_t use = (uint32_t)(g / NBUF);
          if (!mbar_wait<PAIR>(&tempty[buf], (use & 1) ^ 1, abort_flag, p.status, ST_MMA, limit_ns,
                               peer_abort)) {
            go = false;
            break;
          }
          tc_fence_after();
          const uint32_t dst = tmem + buf * TN;
          const int kb_first = kb_lo + c * KC_SLABS;
          const int kb_end = min(kb_hi, kb_first + KC_SLABS);
          for (int kb = kb_first; kb < kb_end; ++kb, ++it) {
            const int s = it % S;
            const uint32_t ph = (it / S) & 1;
            if (!mbar_wait<PAIR>(&full[s], ph, abort_flag, p.status, ST_MMA, limit_ns, peer_abort)) {
              go = false;
              break;
            }
            tc_fence_after();
            // The slab's descriptors (their low words), built once: the K
            // step's are the slab's plus off, the step's bytes >> 4.
            constexpr int RB = C_::ROW_BYTES;
            const uint32_t ah = sdesc_lo(smem_u32(a_hi(s))), al = sdesc_lo(smem_u32(a_pl(s, 1)));
            const uint32_t bh = sdesc_lo(smem_u32(b_hi(s))), bl = sdesc_lo(smem_u32(b_pl(s, 1)));
#pragma unroll
            for (int kk = 0; kk < BK / MMA_K; ++kk) {
              const uint32_t off = (kk * MMA_K * C_::ELEM_BYTES) >> 4;  // 16-byte units along the slab row
              const uint32_t acc = (kb == kb_first && kk == 0) ? 0u : 1u;
              if (C_::FP8) {
                umma_e4m3<CG>(dst, sdesc_of<RB>(ah + off), sdesc_of<RB>(bh + off), idesc, acc);
              } else if (NPROD == 3) {
                umma_bf16<CG>(dst, sdesc_of<RB>(al + off), sdesc_of<RB>(bh + off), idesc, acc);
                umma_bf16<CG>(dst, sdesc_of<RB>(ah + off), sdesc_of<RB>(bl + off), idesc, 1u);
                umma_bf16<CG>(dst, sdesc_of<RB>(ah + off), sdesc_of<RB>(bh + off), idesc, 1u);
              } else if constexpr (NPROD == 6) {
                const uint32_t al2 = sdesc_lo(smem_u32(a_pl(s, 2))), bl2 = sdesc_lo(smem_u32(b_pl(s, 2)));
                // smallest first: lo*hi, hi*lo, mid*mid (2^-17 of hi*hi),
                // mid*hi, hi*mid (2^-9), hi*hi (the lo planes hold mid, the
                // lo2 planes lo)
                umma_bf16<CG>(dst, sdesc_of<RB>(al2 + off), sdesc_of<RB>(bh + off), idesc, acc);
                umma_bf16<CG>(dst, sdesc_of<RB>(ah + off), sdesc_of<RB>(bl2 + off), idesc, 1u);
                umma_bf16<CG>(dst, sdesc_of<RB>(al + off), sdesc_of<RB>(bl + off), idesc, 1u);
                umma_bf16<CG>(dst, sdesc_of<RB>(al + off), sdesc_of<RB>(bh + off), idesc, 1u);
                umma_bf16<CG>(dst, sdesc_of<RB>(ah + off), sdesc_of<RB>(bl + off), idesc, 1u);
                umma_bf16<CG>(dst, sdesc_of<RB>(ah + off), sdesc_of<RB>(bh + off), idesc, 1u);
              } else {
                umma_bf16<CG>(dst, sdesc_of<RB>(ah + off), sdesc_of<RB>(bh + off), idesc, acc);
              }
            }
            umma_commit<CG>(&empty[s]);  // frees the slab (in both CTAs) once read
          }
          if (!go) break;
          umma_commit<CG>(&tfull[buf]);  // chunk complete in buffer buf (both CTAs)
        }
      }
    } else if (CONVERT && (warp == 2 || warp == 3)) {
      // ---- converter: chunks in claim order, four 32-row pieces each, two
      // staging buffers (the next piece's TMA load in flight while this one
      // is converted); lane l converts row l of a piece
      const int w = warp - 2;
      if constexpr (CONVERT && GROUPED)
        cv_convert_batch(cv, cvbuf + w * 2 * CV_PIECE_BYTES, lane, abort_flag);
      else if constexpr (CONVERT)
        cv_convert(cv, cvtab, cvbar + 2 * w, cvbuf + w * 2 * CV_PIECE_BYTES, lane, abort_flag, p.status, limit_ns);
    }
    __syncwarp();
    tc_fence_before();
    cta_barrier_all();  // every role of this CTA is done
    tc_fence_after();
    // Both CTAs of a pair are past their roles before either decides whether
    // to drain: an abort either of them raised (its own flag, or the copy it
    // stored in the peer's) is then seen by both.
    if constexpr (PAIR) cluster_sync_all();
    bool aborted = *abort_flag != 0;
    if constexpr (PAIR) aborted = aborted || ld_cluster_u32(peer_abort) != 0;
    if (aborted) {
      // Drain what was started before returning (bounded waits).
      // Loads: the last S stages either CTA issued (an earlier stage's slot
      // was refilled, so its loads had landed). Both CTAs' loads complete on
      // the leader's barrier, which at issue expects the pair's bytes; the
      // leader squares that with what was issued: a stage only the leader
      // issued counts the peer's bytes as arrived, a stage only the peer
      // issued gets the leader's arrival and expects the peer's bytes. Each
      // such stage then completes once its loads have landed.
      if (warp == 0 && lane == 0 && leader) {
        constexpr uint32_t CTA_BYTES = C_::PLANES * (C_::A_SLAB + C_::B_SLAB);
        const int mine = issued;
        int theirs = mine;
        if constexpr (PAIR) theirs = (int)ld_cluster_u32(mapa_rank(smem_u32((const void*)issued_sh), 1));
        const int hi = max(mine, theirs);
        for (int it = max(0, hi - S); it < hi; ++it) {
          const int s = it % S;
          if constexpr (PAIR) {
            // the bytes of stage it's tile for one CTA: a constant, except
            // in a batch (its issuer's record: ours, or the peer's)
            uint32_t own = CTA_BYTES, peer = CTA_BYTES;
            if constexpr (GROUPED) {
              own = stage_bytes_sh[s];
              peer = ld_cluster_u32(mapa_rank(smem_u32(&stage_bytes_sh[s]), 1));
            }
            if (it < mine && it >= theirs) mbar_complete_tx(&full[s], own);
            else if (it >= mine && it < theirs) mbar_expect_tx(&full[s], peer);
          }
          const uint64_t t0 = globaltimer();
          while (!mbar_try_wait<PAIR>(&full[s], (it / S) & 1)) {
            if (globaltimer() - t0 > WAIT_LIMIT_NS) {
              if (p.status) atomicOr_system(p.status, ST_DRAIN);
              break;
            }
          }
        }
      }
      // MMAs: a last commit by the issuer, after every MMA it issued, arrives
      // on the drain barrier of each CTA (both of a pair) once they are done
      if (warp == 1 && lane == 0) {
        if (leader) umma_commit<CG>(drainbar);
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait<PAIR>(drainbar, 0)) {
          if (globaltimer() - t0 > WAIT_LIMIT_NS) {
            if (p.status) atomicOr_system(p.status, ST_DRAIN);
            break;
          }
        }
      }
    }
    __syncwarp();  // warp 1: the drain of lane 0 ends before the dealloc
    // PAIR: neither CTA leaves (or frees tensor memory) while the other may
    // still arrive on its barriers or the leader's MMAs may read its stages
    if constexpr (PAIR) cluster_sync_all();
    if (warp == 1) {
      tc_fence_after();
      if constexpr (PAIR)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
      else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(RegSplit<MODE, EPI, PAIR, CONVERT>::EPI_R));
    // ---- epilogue: every chunk, tensor memory -> FP32 registers (round to
    // nearest); at the end of a tile, registers -> C, coalesced per column.
    // PAIR: this CTA's tensor memory holds rows rank*128 .. +127 of the tile.
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int h = (warp - EPI_WARP0) >> 2;  // which half of the tile's columns
    int g = 0;
    bool go = true;
    GroupTile nx = fetch(unit);
    for (int t = unit; go && t < num_work; t += num_units) {
      const GroupTile cur = nx;
      nx = fetch(t + num_units);
      const TileView v = view(t, cur);
      const int m_cta = v.m0 + (int)rank * BM;  // first row of this CTA's half
      const int num_chunks = TAIL ? (v.kb1 - v.kb0 + KC_SLABS - 1) / KC_SLABS
                                  : ((v.K + BK - 1) / BK + KC_SLABS - 1) / KC_SLABS;
      // the columns this warp owns: [coff, coff + cols) of the tile
      const int cols = GROUPED ? v.bn / 2 : (h ? C_::COLS1 : C_::COLS0);
      const int coff = GROUPED ? h * (v.bn / 2) : (h ? C_::COLS0 : 0);
      constexpr int ACC = C_::ACC;
      float acc[ACC];
#pragma unroll
      for (int u = 0; u < ACC; ++u) acc[u] = 0.f;
      // FP8: this warp's 128 columns are exactly one 128-wide block of
      // op(B)^T rows and this CTA's tile rows one block of op(A) rows
      static_assert(!C_::FP8 || (C_::COLS0 == FP8_BLOCK && C_::COLS1 == FP8_BLOCK), "one scale block per warp");
      const bool live = v.n0 + coff < v.N && m_cta < v.M;
      const float* sa = nullptr;
      const float* sb = nullptr;
      if (C_::FP8) {
        // (a K half starts at its first slab's scale block)
        sa = p.scaleA + (int64_t)(m_cta / FP8_BLOCK) * p.nkb + (TAIL ? v.kb0 / KC_SLABS : 0);
        sb = p.scaleB + (int64_t)((v.n0 + coff) / FP8_BLOCK) * p.nkb + (TAIL ? v.kb0 / KC_SLABS : 0);
      }
      // FP8: the block scales 32 chunks at a time, lane l holding chunk
      // 32 j + l's (one coalesced load per batch, read by shuffle), the next
      // batch loaded a whole batch ahead
      float sa0 = 0.f, sb0 = 0.f, sa1 = 0.f, sb1 = 0.f;
      if (C_::FP8 && live) {
        if (lane < num_chunks) sa0 = __ldg(sa + lane), sb0 = __ldg(sb + lane);
        if (32 + lane < num_chunks) sa1 = __ldg(sa + 32 + lane), sb1 = __ldg(sb + 32 + lane);
      }
      for (int c = 0; c < num_chunks; ++c, ++g) {
        const int buf = g % NBUF;
        const uint32_t use = (uint32_t)(g / NBUF);
        float scale = 1.f;  // FP8: the chunk's sA * sB
        if (C_::FP8) {
          scale = __shfl_sync(0xffffffffu, sa0, c & 31) * __shfl_sync(0xffffffffu, sb0, c & 31);
          if ((c & 31) == 31) {
            sa0 = sa1;
            sb0 = sb1;
            if (live && c + 33 + lane < num_chunks) sa1 = __ldg(sa + c + 33 + lane), sb1 = __ldg(sb + c + 33 + lane);
          }
        }
        // Lane 0 alone waits (bounded) and the warp takes its outcome, so no
        // warp splits between a lane that saw the chunk and one that saw the
        // abort flag; after a success the other lanes observe the completed
        // phase, which their first poll returns.
        int seen = 0;
        if (lane == 0)
          seen = mbar_wait<PAIR>(&tfull[buf], use & 1, abort_flag, p.status, ST_EPILOGUE, wait_limit(p), peer_abort);
        if (!__shfl_sync(0xffffffffu, seen, 0)) {
          go = false;
          break;
        }
        for (int n = 0; n < (1 << 20) && !mbar_try_wait<PAIR>(&tfull[buf], use & 1); ++n) {
        }
        tc_fence_after();
        __syncwarp();
        const uint32_t src = tmem + (static_cast<uint32_t>(q * 32) << 16) + buf * TN + coff;
        if constexpr (ACC <= 96) {
          // every 32-column load of this warp in flight before one wait
          uint32_t r[ACC / 32][32];
#pragma unroll
          for (int i = 0; i < ACC / 32; ++i)
            if (i * 32 < cols) tmem_ld_x32_issue(src + i * 32, r[i]);
#pragma unroll
          for (int i = 0; i < ACC / 32; ++i)
            if (i * 32 < cols) tmem_wait_ld_into(r[i]);
#pragma unroll
          for (int i = 0; i < ACC / 32; ++i) {
            if (i * 32 < cols) {
#pragma unroll
              for (int u = 0; u < 32; u += 2) {
                ffma2(acc[i * 32 + u], acc[i * 32 + u + 1], scale, r[i][u], r[i][u + 1]);
              }
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < ACC / 32; i += 2) {
            // 64 columns per step, two loads in flight (cols is a multiple of
            // 32; a 32-column warp share takes the single-load path)
            if (i * 32 + 32 < cols) {
              uint32_t r[32], r2[32];
              tmem_ld_2x32(src + i * 32, src + i * 32 + 32, r, r2);
#pragma unroll
              for (int u = 0; u < 32; u += 2) {
                ffma2(acc[i * 32 + u], acc[i * 32 + u + 1], scale, r[u], r[u + 1]);
              }
#pragma unroll
              for (int u = 0; u < 32; u += 2) {
                ffma2(acc[i * 32 + 32 + u], acc[i * 32 + 33 + u], scale, r2[u], r2[u + 1]);
              }
            } else if (i * 32 < cols) {
              uint32_t r[32];
              tmem_ld_x32(src + i * 32, r);
#pragma unroll
              for (int u = 0; u < 32; u += 2) {
                ffma2(acc[i * 32 + u], acc[i * 32 + u + 1], scale, r[u], r[u + 1]);
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if constexpr (PAIR)
            mbar_arrive_cluster(mapa_rank(smem_u32(&tempty[buf]), 0));  // the leader's barrier
          else
            mbar_arrive(&tempty[buf]);
        }
      }
      if (!go) break;
      if (TAIL && v.part >= 0) {
        // tail split: this half's partial sums out (per thread its ACC
        // columns, coalesced across the warp), then one arrival per warp;
        // the second half to arrive adds the other's and writes C
        constexpr int RANKS = PAIR ? 2 : 1;
        const int wi = warp - EPI_WARP0;
        const int64_t slot = ((int64_t)(v.tail * 2 + v.part) * RANKS + (int)rank) * EPI_WARPS + wi;
        const int64_t other = slot + (v.part ? -1 : 1) * (int64_t)RANKS * EPI_WARPS;
        int* cnt = reinterpret_cast<int*>(p.split_ws + (int64_t)n_split * 2 * RANKS * EPI_WARPS * ACC * 32) +
                   ((int64_t)v.tail * RANKS + (int)rank) * EPI_WARPS + wi;
        float* mine = p.split_ws + slot * (ACC * 32) + lane;
#pragma unroll
        for (int u = 0; u < ACC; ++u) __stcg(mine + u * 32, acc[u]);
        __threadfence();
        __syncwarp();
        int arrived = 0;
        if (lane == 0) arrived = atomicAdd(cnt, 1);
        arrived = __shfl_sync(0xffffffffu, arrived, 0);
        if (arrived == 0) continue;  // the other half writes C
        __threadfence();
        const float* theirs = p.split_ws + other * (ACC * 32) + lane;
#pragma unroll
        for (int u = 0; u < ACC; ++u) acc[u] += __ldcg(theirs + u * 32);
      }
      if (!GROUPED && (EPI == 2 || p.beta != 0.f)) {
        // The next tile's epilogue inputs (old C when beta != 0, H for the
        // tanh adjoint) are fetched into L2 now, while its MMAs run: its
        // loads then wait on L2 rather than on DRAM.
        const int tn = t + num_units;
        if (tn < num_work) {
          int nm0, nn0, npart;
          tile_coords(TAIL ? work_tile(tn, &npart) : tn, tiles_m, tiles_n, TM, TN, &nm0, &nn0);
          const int r0 = nm0 + (int)rank * BM + q * 32;  // this warp's 32 rows there
          const int c0 = nn0 + coff;
          if (r0 < p.M && c0 < p.N) {
            const int nc = min(cols, p.N - c0);
            for (int u = lane; u < nc; u += 32) {
              if (p.beta != 0.f) prefetch_l2(p.C + r0 + (int64_t)(c0 + u) * p.ldc);
              if (EPI == 2) prefetch_l2(p.aux + r0 + (int64_t)(c0 + u) * p.ldaux);
            }
          }
        }
      }
      const int row = m_cta + q * 32 + lane;
      const int col0 = v.n0 + coff;
      if (row < v.M) {
        // C in groups of CGRP columns: all loads of old C values first, so
        // their DRAM round trips overlap, then the stores (streaming hints:
        // C is touched once and should not displace operand panels in L2)
        float* cp = v.C + row + (int64_t)col0 * v.ldc;
        const int ncols = min(cols, v.N - col0);
        // 16 columns per group (8 measured 1% slower at 8192, 32 no faster);
        // 8 for the tanh adjoint, which also reads H (4 made the chain's
        // training step 5% slower, 16 columns of H alone no faster)
        constexpr int CGRP = EPI == 2 ? 8 : 16;
#pragma unroll
        for (int u0 = 0; u0 < ACC; u0 += CGRP) {
          float old[CGRP];
          if (v.beta != 0.f) {
#pragma unroll
            for (int u = 0; u < CGRP; ++u) old[u] = (u0 + u < ncols) ? __ldcs(cp + (int64_t)(u0 + u) * v.ldc) : 0.f;
          }
          float hx[EPI == 2 ? CGRP : 1];
          if (EPI == 2) {
            const float* hp = p.aux + row + (int64_t)col0 * p.ldaux;
#pragma unroll
            for (int u = 0; u < CGRP; ++u) hx[u] = (u0 + u < ncols) ? __ldcs(hp + (int64_t)(u0 + u) * p.ldaux) : 0.f;
            // the next group's H into L1 while this group is computed and
            // stored (no registers: held one group ahead, the loads spilled;
            // not in the FP8 leaf, which spilled with the prefetches too)
            if (!C_::FP8 && u0 + CGRP < ACC) {
#pragma unroll
              for (int u = 0; u < CGRP; ++u)
                if (u0 + CGRP + u < ncols) prefetch_l1(hp + (int64_t)(u0 + CGRP + u) * p.ldaux);
            }
          }
          // C, the forwarded planes and, for the tanh stages (EPI != 0),
          // C's row planes. The plain leaf keeps its own loop: ptxas spills
          // its epilogue when that loop takes the blocked form below.
          constexpr bool ROWS = !GROUPED && !C_::FP8 && EPI != 0;
          if constexpr (!ROWS) {
#pragma unroll
            for (int u = 0; u < CGRP; ++u) {
              if (u0 + u < ncols) {
                float x = (v.beta == 0.f) ? v.alpha * acc[u0 + u] : fmaf(v.alpha, acc[u0 + u], v.beta * old[u]);
                if (EPI == 1) x = tanhf(x);
                if (EPI == 2) x = x * (1.f - hx[u] * hx[u]);
                if (GROUPED || C_::FP8 || !p.planes_only) __stcs(cp + (int64_t)(u0 + u) * v.ldc, x);
                if (!GROUPED && !C_::FP8 && p.fwd_hi) {
                  // the next stage's operand planes of this output (a warp
                  // writes 32 consecutive K elements of one plane row)
                  const int64_t o = (int64_t)(col0 + u0 + u) * p.fwd_kp + row;
                  const __nv_bfloat16 h = __float2bfloat16_rn(x);
                  p.fwd_hi[o] = h;
                  if (NPROD == 3) p.fwd_lo[o] = __float2bfloat16_rn(x - __bfloat162float(h));
                }
              }
            }
          } else {
            // 8 columns at a time, one 16-byte store per row plane and row
#pragma unroll
            for (int j = 0; j < CGRP / 8; ++j) {
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                float x2[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  const int u = 8 * j + 2 * e + h;
                  x2[h] = 0.f;
                  if (u0 + u < ncols) {
                    float x = (v.beta == 0.f) ? v.alpha * acc[u0 + u] : fmaf(v.alpha, acc[u0 + u], v.beta * old[u]);
                    if (EPI == 1) x = tanhf(x);
                    if (EPI == 2) x = x * (1.f - hx[u] * hx[u]);
                    x2[h] = x;
                    if (!p.planes_only) __stcs(cp + (int64_t)(u0 + u) * v.ldc, x);  // (ROWS variants only)
                    if (!GROUPED && !C_::FP8 && p.fwd_hi) {
                      // the next stage's operand planes of this output (a warp
                      // writes 32 consecutive K elements of one plane row)
                      const int64_t o = (int64_t)(col0 + u0 + u) * p.fwd_kp + row;
                      const __nv_bfloat16 hv = __float2bfloat16_rn(x);
                      p.fwd_hi[o] = hv;
                      if (NPROD == 3) p.fwd_lo[o] = __float2bfloat16_rn(x - __bfloat162float(hv));
                    }
                  }
                }
                const __nv_bfloat162 hh = __floats2bfloat162_rn(x2[0], x2[1]);
                hw[e] = *reinterpret_cast<const uint32_t*>(&hh);
                if (NPROD == 3) {
                  const __nv_bfloat162 ll = __floats2bfloat162_rn(x2[0] - __low2float(hh), x2[1] - __high2float(hh));
                  lw[e] = *reinterpret_cast<const uint32_t*>(&ll);
                }
              }
              const int c = col0 + u0 + 8 * j;  // a multiple of 8: 16-byte aligned
              if (p.row_hi && c < v.N) {
                // columns past N are zeros inside the plane row's padding
                const int64_t o = (int64_t)row * p.row_kp + c;
                *reinterpret_cast<uint4*>(p.row_hi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                if (NPROD == 3) {
                  // the lo plane starts at the hi plane's 256-byte-aligned end
                  const int64_t lo = (((int64_t)p.M * p.row_kp * 2 + 255) & ~(int64_t)255) / 2;
                  *reinterpret_cast<uint4*>(p.row_hi + lo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
                }
              }
            }
          }
        }
      }
    }
    tc_fence_before();
    cta_barrier_all();
    if constexpr (PAIR) {  // the control warpgroup's two cluster barriers (before and after its drain)
      cluster_sync_all();
      cluster_sync_all();
    }
  }
}

// A wait that nothing satisfies: the bounded wait the leaf kernels use must
// give up after limit_ns, record ST_SELFTEST in the status word and let the
// kernel return (no copy, MMA or tensor memory is involved).
__global__ void wait_selftest(int* status, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&bar, 0, &abort_flag, status, ST_SELFTEST, limit_ns);
  __syncthreads();
}

// ---- host side ---------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// K-major operand plane: rows x K elements of `elem_bytes` bytes, row stride
// Kp elements; TMA box of one slab row (row_bytes, 64 or 128, with the
// matching swizzle) x box_rows rows.
bool encode_plane(CUtensorMap* map, const void* base, int rows, int K, int Kp, int box_rows, int elem_bytes,
                  int row_bytes, std::string* err) {
  auto enc = get_encoder();
  if (!enc) {
    *err = "cuTensorMapEncodeTiled is not available from the driver";
    return false;
  }
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * elem_bytes};
  cuuint32_t box[2] = {(cuuint32_t)(row_bytes / elem_bytes), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[160];
    snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d) for a %d x %d plane", (int)r, rows, K);
    *err = buf;
    return false;
  }
  return true;
}

// Per-device caches: kernel attributes (cudaFuncSetAttribute applies to the
// device current when it is called), occupancy and the SM count are looked
// up once per device and kept per device, so launches on several devices
// of one process each see their own device's values. Entries are atomics:
// two threads that race fill in the same value. A device numbered beyond
// the cache (or none current) is looked up at every call.
constexpr int kMaxDevices = 64;
int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  return dev;
}
inline bool cached_device(int dev) { return dev >= 0 && dev < kMaxDevices; }

// FP32 operand with rows contiguous (element (r, k) at X[r + k * ld]) for
// the in-leaf conversion: a box of 32 rows x 64 K, no swizzle (the
// converter reads the staged piece column by column).
bool encode_fp32_rows(CUtensorMap* map, const float* X, int64_t ld, int rows, int K, std::string* err) {
  auto enc = get_encoder();
  if (!enc) {
    *err = "cuTensorMapEncodeTiled is not available from the driver";
    return false;
  }
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)K};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)CV_PIECE, (cuuint32_t)CV_BK};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[160];
    snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d) for a %d x %d FP32 operand", (int)r, rows, K);
    *err = buf;
    return false;
  }
  return true;
}

int num_sms() {
  static std::atomic<int> cache[kMaxDevices];
  const int dev = current_device();
  int n = cached_device(dev) ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (n == 0) {
    if (dev < 0 || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    if (cached_device(dev)) cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Which leaves of a single instance run on CTA pairs (256 x 256 tiles,
// cta_group::2) rather than on single CTAs (128 x 256 tiles). Measured at
// M = N = K = 8192 and 16384: pairs make plain BF16 (one accumulation per
// tile) 5-10% faster; BF16x3 on pairs with 128-byte slab rows is 4% faster
// than on single CTAs with 64-byte rows (1.90 vs 1.98 ms at 8192; with
// 64-byte rows on pairs, or 128-byte rows in two stages on single CTAs, it
// is not faster); FP8, which hands a tensor-memory buffer between the MMA
// and epilogue warps every 128 K, runs 3% slower on pairs (2.2x slower
// when the peer released buffers with a cluster-scope release). So BF16
// and BF16x3 run on pairs, FP8 on single CTAs.
constexpr bool pair_for_mode(int mode) { return mode == 1 || mode == 3 || mode == 6; }

// Workspace layout of a mode: operand planes (and FP8 block scales), then
// the tail split's region where the pairs' tiles call for one.
struct WsLayout {
  int64_t Kp = 0;  // row stride of the planes, in elements (16-byte rows)
  size_t a_hi = 0, a_lo = 0, b_hi = 0, b_lo = 0, sa = 0, sb = 0, total = 0;
  size_t a_lo2 = 0, b_lo2 = 0;  // BF16x6: the third parts
  int nkb = 0;     // FP8: scale blocks along K
  size_t planes = 0;                   // end of the planes: the least a launch needs
  size_t split = 0, split_bytes = 0;   // the tail split's partial sums and counters
  size_t conv = 0, conv_bytes = 0;     // BF16x3: the in-leaf conversion's chunk flags and counter
};

// Bytes of a tail split of n tiles: per tile, K half, CTA and epilogue warp
// ACC x 32 FP32 partial sums, then per tile, CTA and warp one counter.
size_t split_sums_bytes(int n, int ranks, int acc) {
  return (size_t)n * 2 * ranks * EPI_WARPS * acc * 32 * sizeof(float);
}
size_t split_region_bytes(int n, int ranks, int acc) {
  return align256(split_sums_bytes(n, ranks, acc)) + align256((size_t)n * ranks * EPI_WARPS * sizeof(int));
}
WsLayout ws_layout(const SgemmDesc& d, int mode) {
  WsLayout L;
  const int eb = mode == 8 ? 1 : 2;
  L.Kp = (d.K + 16 / eb - 1) / (16 / eb) * (16 / eb);
  const size_t ap = align256((size_t)d.M * L.Kp * eb), bp = align256((size_t)d.N * L.Kp * eb);
  size_t off = 0;
  L.a_hi = off; off += ap;
  if (mode == 3 || mode == 6) { L.a_lo = off; off += ap; }
  if (mode == 6) { L.a_lo2 = off; off += ap; }
  L.b_hi = off; off += bp;
  if (mode == 3 || mode == 6) { L.b_lo = off; off += bp; }
  if (mode == 6) { L.b_lo2 = off; off += bp; }
  if (mode == 8) {
    L.nkb = (int)((d.K + FP8_BLOCK - 1) / FP8_BLOCK);
    L.sa = off; off += align256((size_t)((d.M + FP8_BLOCK - 1) / FP8_BLOCK) * L.nkb * 4);
    L.sb = off; off += align256((size_t)((d.N + FP8_BLOCK - 1) / FP8_BLOCK) * L.nkb * 4);
  }
  L.planes = off;
  if (pair_for_mode(mode)) {
    // the tail split's region, for the pairs the GPU runs at once
    using P = Cfg<1, true>;
    static_assert(Cfg<3, true>::BK == P::BK && Cfg<3, true>::ACC == P::ACC && Cfg<6, true>::ACC == P::ACC,
                  "one split layout for the pair tiers");
    const int bk = mode == 6 ? Cfg<6, true>::BK : P::BK;  // the K slab the leaf counts in
    const int64_t tiles = ((d.M + 2 * BM - 1) / (2 * BM)) * ((d.N + P::TN - 1) / P::TN);
    const int n = tiles <= INT32_MAX ? tail_split_tiles((int)tiles, num_sms() / 2, (int)((d.K + bk - 1) / bk)) : 0;
    if (n > 0) {
      L.split = off;
      L.split_bytes = split_region_bytes(n, 2, P::ACC);
      off += L.split_bytes;
    }
  }
  if (mode == 3) {
    // one flag per 128-row block and 64-element slab of each operand (a
    // block's row of flags padded to 4), one count per block, and the claim
    // counter
    const int64_t kb4 = ((d.K + CV_BK - 1) / CV_BK + 3) / 4 * 4;
    const int64_t blocks = (d.M + CV_ROWS - 1) / CV_ROWS + (d.N + CV_ROWS - 1) / CV_ROWS;
    L.conv = off;
    L.conv_bytes = align256((size_t)(blocks * kb4 + blocks + 1) * sizeof(int));
    off += L.conv_bytes;
  }
  L.total = off;
  return L;
}

// The planes of one operand of `rows` rows (a plane cache entry): hi, then
// lo (BF16x3), then the block scales (FP8), each 256-byte aligned.
OperandLayout operand_layout(int64_t rows, int64_t K, int mode) {
  OperandLayout L;
  const int eb = mode == 8 ? 1 : 2;
  const int64_t Kp = (K + 16 / eb - 1) / (16 / eb) * (16 / eb);
  const size_t plane = align256((size_t)rows * Kp * eb);
  size_t off = plane;
  if (mode == 3 || mode == 6) {
    L.lo = off;
    off += plane;
  }
  if (mode == 6) {
    L.lo2 = off;
    off += plane;
  }
  if (mode == 8) {
    L.scales = off;
    off += align256((size_t)((rows + FP8_BLOCK - 1) / FP8_BLOCK) * ((K + FP8_BLOCK - 1) / FP8_BLOCK) * 4);
  }
  L.total = off;
  return L;
}

template <int NPROD>
cudaError_t launch_split(const float* X, int64_t ld, bool mmajor, int rows, int K, int Kp,
                         __nv_bfloat16* hi, __nv_bfloat16* lo, __nv_bfloat16* lo2, cudaStream_t s) {
  if (rows == 0 || K == 0) return cudaSuccess;
  if (mmajor) {
    dim3 grid((rows + SPLIT_TR - 1) / SPLIT_TR, (Kp + SPLIT_TK - 1) / SPLIT_TK);
    split_mmajor<NPROD><<<grid, 256, 0, s>>>(X, ld, rows, K, Kp, hi, lo, lo2);
  } else {
    int64_t tasks = (int64_t)rows * (Kp / 8);
    int64_t blocks = (tasks + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    split_kmajor<NPROD><<<(unsigned)blocks, 256, 0, s>>>(X, ld, rows, K, Kp, hi, lo, lo2);
  }
  return cudaGetLastError();
}

cudaError_t launch_quant(const float* X, int64_t ld, bool mmajor, int rows, int K, int Kp, uint8_t* q,
                         float* scales, int nkb, cudaStream_t s) {
  if (rows == 0 || K == 0) return cudaSuccess;
  // float4 loads need 16-byte aligned groups: base aligned and ld % 4 == 0
  const bool vec = (reinterpret_cast<uintptr_t>(X) & 15u) == 0 && ld % 4 == 0;
  dim3 grid((rows + FP8_BLOCK - 1) / FP8_BLOCK, nkb);
  if (mmajor) {
    quant_fp8<false, false><<<grid, QTHREADS, 0, s>>>(X, ld, rows, K, Kp, q, scales, nkb);
  } else {
    if (vec) quant_fp8<true, true><<<grid, QTHREADS, 0, s>>>(X, ld, rows, K, Kp, q, scales, nkb);
    else quant_fp8<true, false><<<grid, QTHREADS, 0, s>>>(X, ld, rows, K, Kp, q, scales, nkb);
  }
  return cudaGetLastError();
}

// The leaf's register split (setmaxnreg) moves registers between the
// warpgroups of a block; it only balances when the block was launched with
// LAUNCH_REGS registers per thread. A build that gave the kernel fewer would
// make setmaxnreg.inc wait for registers that never come, so it is refused.
template <typename Kern>
cudaError_t check_register_split(Kern* kernel) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  if (a.numRegs < LAUNCH_REGS || a.maxThreadsPerBlock < THREADS) return cudaErrorInvalidConfiguration;
  return cudaSuccess;
}

// The single-instance leaf, persistent: PAIR runs clusters of 2, one cluster
// per 256 x 256 tile at a time, as many clusters as fit on the GPU at once;
// otherwise one CTA per SM. *grid_ctas returns the CTAs launched.
// The tail split of a launch over `units` units: kept when this variant has
// it, the tiles, units and K call for it and split_cap bytes hold its
// region (its counters zeroed on the stream here), else turned off.
template <int MODE, int EPI, bool PAIR>
cudaError_t tail_setup(TcParams& prm, int tiles, int units, size_t split_cap, int split_as, cudaStream_t s) {
  using C_ = Cfg<MODE, PAIR>;
  constexpr int RANKS = PAIR ? 2 : 1;
  const bool variant = tail_split_variant(MODE, EPI, false) &&
                       (split_as < 0 || tail_split_variant(MODE, split_as, false));
  const int n = (variant && prm.split_ws)
                    ? tail_split_tiles(tiles, units, (prm.K + C_::BK - 1) / C_::BK)
                    : 0;
  if (n == 0 || split_region_bytes(n, RANKS, C_::ACC) > split_cap) {
    prm.split_ws = nullptr;
    return cudaSuccess;
  }
  return cudaMemsetAsync(reinterpret_cast<uint8_t*>(prm.split_ws) + split_sums_bytes(n, RANKS, C_::ACC), 0,
                         (size_t)n * RANKS * EPI_WARPS * sizeof(int), s);
}

// The pairs a launch of this leaf variant runs at once (the clusters the
// GPU holds), looked up per device; sets the kernel's attributes first.
template <int MODE, int EPI, bool CONVERT>
cudaError_t pair_units(int* units) {
  using C_ = Cfg<MODE, true>;
  auto kernel = sgemm_tc<MODE, EPI, false, true, CONVERT>;
  constexpr uint32_t smem = C_::SMEM_BYTES + (CONVERT ? CV_SMEM : 0);
  const int dev = current_device();
  static std::atomic<int> max_clusters_of[kMaxDevices];
  int n = cached_device(dev) ? max_clusters_of[dev].load(std::memory_order_acquire) : 0;
  if (n == 0) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = check_register_split(kernel);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(2 * num_sms());
    e = cudaOccupancyMaxActiveClusters(&n, kernel, &cfg);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    if (cached_device(dev)) max_clusters_of[dev].store(n, std::memory_order_release);
  }
  *units = n;
  return cudaSuccess;
}

template <int MODE, int EPI, bool PAIR, bool CONVERT = false>
cudaError_t launch_leaf(const CUtensorMap* maps, TcParams prm, int tiles, size_t split_cap, int split_as,
                        cudaStream_t s, int* grid_ctas, const LaunchHooks* hooks, const ConvParams& cvp) {
  using C_ = Cfg<MODE, PAIR>;
  static_assert(!CONVERT || PAIR, "in-leaf conversion on pairs");
  auto kernel = sgemm_tc<MODE, EPI, false, PAIR, CONVERT>;
  if constexpr (!PAIR) {
    const int dev = current_device();
    static std::atomic<bool> attr_set[kMaxDevices];
    if (!cached_device(dev) || !attr_set[dev].load(std::memory_order_acquire)) {
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C_::SMEM_BYTES);
      if (e == cudaSuccess) e = check_register_split(kernel);
      if (e != cudaSuccess) return e;
      if (cached_device(dev)) attr_set[dev].store(true, std::memory_order_release);
    }
    const int grid = std::max(1, std::min(tiles, num_sms()));
    *grid_ctas = grid;
    cudaError_t e = tail_setup<MODE, EPI, PAIR>(prm, tiles, grid, split_cap, split_as, s);
    if (e != cudaSuccess) return e;
    hook_begin(hooks, s);
    kernel<<<grid, THREADS, C_::SMEM_BYTES, s>>>(maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], prm,
                                                  GroupParams{nullptr, nullptr, 0}, cvp);
    e = cudaGetLastError();
    hook_end(hooks, s);
    return e;
  } else {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = C_::SMEM_BYTES + (CONVERT ? CV_SMEM : 0);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int max_clusters = 0;
    if (cudaError_t e = pair_units<MODE, EPI, CONVERT>(&max_clusters); e != cudaSuccess) return e;
    const int clusters = std::max(1, std::min(tiles, max_clusters));
    cfg.gridDim = dim3(2 * clusters);
    *grid_ctas = 2 * clusters;
    cudaError_t e = tail_setup<MODE, EPI, PAIR>(prm, tiles, clusters, split_cap, split_as, s);
    if (e != cudaSuccess) return e;
    hook_begin(hooks, s);
    e = cudaLaunchKernelEx(&cfg, kernel, maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], prm,
                           GroupParams{nullptr, nullptr, 0}, cvp);
    hook_end(hooks, s);
    return e;
  }
}

template <int MODE>
cudaError_t run_tc(const SgemmDesc& d, void* ws, size_t ws_bytes, const DeviceStatus& st, cudaStream_t s,
                   KernelReport* rep, std::string* err, const LaunchHooks* hooks, const Epilogue& epi,
                   const OperandPlanes& pa, const OperandPlanes& pb) {
  constexpr bool PAIR = pair_for_mode(MODE);
  constexpr int TM = PAIR ? 2 * BM : BM;
  using C_ = Cfg<MODE, PAIR>;
  constexpr int NPROD = MODE == 3 ? 3 : MODE == 6 ? 6 : 1;
  const int M = (int)d.M, N = (int)d.N, K = (int)d.K;
  if (MODE == 6 && (epi.kind != 0 || epi.fwd || epi.rows)) {
    *err = "the BF16X6 tier runs the plain sgemm leaf (no merged elementwise leaf, no forwarded planes)";
    return cudaErrorInvalidValue;
  }
  const WsLayout L = ws_layout(d, MODE);
  const int Kp = (int)L.Kp;
  uint8_t* w = static_cast<uint8_t*>(ws);
  void* ah = w + L.a_hi;
  void* al = w + L.a_lo;
  void* bh = w + L.b_hi;
  void* bl = w + L.b_lo;
  void* al2 = w + L.a_lo2;
  void* bl2 = w + L.b_lo2;
  float* sa = reinterpret_cast<float*>(w + L.sa);
  float* sb = reinterpret_cast<float*>(w + L.sb);
  if (pa.base) {  // op(A)'s planes live in the plane cache
    const OperandLayout O = operand_layout(M, K, MODE);
    uint8_t* b = static_cast<uint8_t*>(pa.base);
    ah = b + O.hi;
    al = b + O.lo;
    al2 = b + O.lo2;
    sa = reinterpret_cast<float*>(b + O.scales);
  }
  if (pb.base) {
    const OperandLayout O = operand_layout(N, K, MODE);
    uint8_t* b = static_cast<uint8_t*>(pb.base);
    bh = b + O.hi;
    bl = b + O.lo;
    bl2 = b + O.lo2;
    sb = reinterpret_cast<float*>(b + O.scales);
  }
  int kernels = 0;
  cudaError_t e = cudaSuccess;
  const int tiles = ((M + TM - 1) / TM) * ((N + C_::TN - 1) / C_::TN);
  // In-leaf conversion (ConvParams): the plain BF16x3 leaf writing its own
  // planes into the workspace, for operands whose rows are contiguous and
  // TMA-readable (16-byte aligned base and leading dimension), on launches
  // that fill the GPU with at least 32 pair tiles and whose grouped order
  // has at most CV_MAX_ROUNDS rounds.
  ConvParams cvp;
  memset(&cvp, 0, sizeof cvp);
  bool convert = false;
  if constexpr (MODE == 3) {
    int units = 0;
    convert = !epi.separate_split && epi.kind == 0 && !epi.fwd && !epi.rows && !pa.base && !pb.base && K > 0 &&
              !d.transA && d.transB && (reinterpret_cast<uintptr_t>(d.A) & 15u) == 0 &&
              (reinterpret_cast<uintptr_t>(d.B) & 15u) == 0 && d.lda % 4 == 0 && d.ldb % 4 == 0 && tiles >= 32 &&
              L.conv_bytes && ws_bytes >= L.conv + L.conv_bytes;
    int pre_rows[2] = {0, 0};
    if (convert) {
      if ((e = pair_units<3, 0, true>(&units)) != cudaSuccess) return e;
      const int U = std::max(1, std::min(tiles, units));
      // the first round's row tiles (rt * gn0 < U) and column tiles (first
      // used by a tile < U), as rows of op(A) and of op(B)^T
      const int tiles_m = (M + TM - 1) / TM, tiles_n = (N + C_::TN - 1) / C_::TN;
      const int gn0 = std::min(GROUP_N, tiles_n);
      int ct = 0;
      while (ct < tiles_n && (ct / GROUP_N) * GROUP_N * tiles_m + ct % GROUP_N < U) ++ct;
      pre_rows[0] = std::min(M, std::min(tiles_m, (U + gn0 - 1) / gn0) * TM);
      pre_rows[1] = std::min(N, ct * C_::TN);
      // worth it only when later rounds hold most of the operands
      convert = (tiles + U - 1) / U <= CV_MAX_ROUNDS && 2 * ((int64_t)pre_rows[0] + pre_rows[1]) <= (int64_t)M + N;
    }
    if (convert) {
      if (!encode_fp32_rows(&cvp.src[0], d.A, d.lda, M, K, err) ||
          !encode_fp32_rows(&cvp.src[1], d.B, d.ldb, N, K, err))
        return cudaErrorInvalidValue;
      cvp.hi[0] = static_cast<__nv_bfloat16*>(ah);
      cvp.lo[0] = static_cast<__nv_bfloat16*>(al);
      cvp.hi[1] = static_cast<__nv_bfloat16*>(bh);
      cvp.lo[1] = static_cast<__nv_bfloat16*>(bl);
      cvp.rows[0] = M;
      cvp.rows[1] = N;
      cvp.blocks[0] = (M + CV_ROWS - 1) / CV_ROWS;
      cvp.blocks[1] = (N + CV_ROWS - 1) / CV_ROWS;
      cvp.Kp = Kp;
      cvp.num_kb = (K + CV_BK - 1) / CV_BK;
      cvp.kb_stride = (cvp.num_kb + 3) / 4 * 4;
      cvp.flags = reinterpret_cast<int*>(w + L.conv);
      cvp.done = cvp.flags + (int64_t)(cvp.blocks[0] + cvp.blocks[1]) * cvp.kb_stride;
      cvp.claim = cvp.done + (cvp.blocks[0] + cvp.blocks[1]);
      cvp.pre[0] = (pre_rows[0] + CV_ROWS - 1) / CV_ROWS;
      cvp.pre[1] = (pre_rows[1] + CV_ROWS - 1) / CV_ROWS;
      // every flag and the claim counter start at zero in each launch
      if ((e = cudaMemsetAsync(w + L.conv, 0, L.conv_bytes, s)) != cudaSuccess) return e;
      // the first round's rows by the split kernel, before the leaf
      if ((e = launch_split<3>(d.A, d.lda, true, pre_rows[0], K, Kp, static_cast<__nv_bfloat16*>(ah),
                               static_cast<__nv_bfloat16*>(al), nullptr, s)) != cudaSuccess)
        return e;
      if ((e = launch_split<3>(d.B, d.ldb, true, pre_rows[1], K, Kp, static_cast<__nv_bfloat16*>(bh),
                               static_cast<__nv_bfloat16*>(bl), nullptr, s)) != cudaSuccess)
        return e;
      kernels += 2;
    }
  }
  if (K > 0 && !convert) {
    // op(A) rows are contiguous when A is not transposed; op(B)'s N rows when B is
    if (!pa.ready) {
      if (C_::FP8)
        e = launch_quant(d.A, d.lda, !d.transA, M, K, Kp, static_cast<uint8_t*>(ah), sa, L.nkb, s);
      else
        e = launch_split<NPROD>(d.A, d.lda, !d.transA, M, K, Kp, static_cast<__nv_bfloat16*>(ah),
                                static_cast<__nv_bfloat16*>(al), static_cast<__nv_bfloat16*>(al2), s);
      if (e != cudaSuccess) return e;
      if (pa.converted) cudaEventRecord(pa.converted, s);
      kernels += 1;
    }
    if (!pb.ready) {
      if (C_::FP8)
        e = launch_quant(d.B, d.ldb, d.transB != 0, N, K, Kp, static_cast<uint8_t*>(bh), sb, L.nkb, s);
      else
        e = launch_split<NPROD>(d.B, d.ldb, d.transB != 0, N, K, Kp, static_cast<__nv_bfloat16*>(bh),
                                static_cast<__nv_bfloat16*>(bl), static_cast<__nv_bfloat16*>(bl2), s);
      if (e != cudaSuccess) return e;
      if (pb.converted) cudaEventRecord(pb.converted, s);
      kernels += 1;
    }
  }
  // A hi, A lo, B hi, B lo, A lo2, B lo2 (planes a mode does not have repeat hi)
  alignas(64) CUtensorMap maps[6];
  memset(maps, 0, sizeof maps);
  if (K > 0) {
    // a CTA loads 128 rows of A and B_ROWS of B (PAIR: 128 of the tile's 256)
    if (!encode_plane(&maps[0], ah, M, K, Kp, BM, C_::ELEM_BYTES, C_::ROW_BYTES, err) ||
        !encode_plane(&maps[2], bh, N, K, Kp, C_::B_ROWS, C_::ELEM_BYTES, C_::ROW_BYTES, err))
      return cudaErrorInvalidValue;
    if (NPROD >= 3) {
      if (!encode_plane(&maps[1], al, M, K, Kp, BM, 2, C_::ROW_BYTES, err) ||
          !encode_plane(&maps[3], bl, N, K, Kp, C_::B_ROWS, 2, C_::ROW_BYTES, err))
        return cudaErrorInvalidValue;
    } else {
      maps[1] = maps[0];
      maps[3] = maps[2];
    }
    if (NPROD == 6) {
      if (!encode_plane(&maps[4], al2, M, K, Kp, BM, 2, C_::ROW_BYTES, err) ||
          !encode_plane(&maps[5], bl2, N, K, Kp, C_::B_ROWS, 2, C_::ROW_BYTES, err))
        return cudaErrorInvalidValue;
    } else {
      maps[4] = maps[0];
      maps[5] = maps[2];
    }
  }
  TcParams prm{M, N, K, 0, d.C, d.ldc, d.alpha, d.beta, sa, sb, L.nkb, 0, st.dev, epi.aux, epi.ldaux,
               nullptr, nullptr, nullptr, nullptr, 0};
  if (epi.rows && !C_::FP8) {
    // the planes of C with rows of C as operand rows: rows = M, row length N
    const OperandLayout F = operand_layout(M, N, MODE);
    uint8_t* f = static_cast<uint8_t*>(epi.rows);
    prm.row_hi = reinterpret_cast<__nv_bfloat16*>(f + F.hi);
    prm.row_kp = (int)((N + 7) / 8 * 8);
    if (MODE == 3 && F.lo != align256((size_t)M * prm.row_kp * 2)) return cudaErrorInvalidValue;
  }
  prm.planes_only = (epi.planes_only && !C_::FP8 && (epi.fwd || epi.rows)) ? 1 : 0;
  prm.wait_limit_us = st.wait_limit_us;
  if (epi.fwd && !C_::FP8) {
    // the planes of C as op(B) of a leaf with K = M: rows = N, row length M
    const OperandLayout F = operand_layout(N, M, MODE);
    uint8_t* f = static_cast<uint8_t*>(epi.fwd);
    prm.fwd_hi = reinterpret_cast<__nv_bfloat16*>(f + F.hi);
    prm.fwd_lo = reinterpret_cast<__nv_bfloat16*>(f + F.lo);
    prm.fwd_kp = (int)((M + 7) / 8 * 8);
  }
  // the tail split's region, when the workspace holds it (the launch decides)
  size_t split_cap = 0;
  if (L.split_bytes && ws_bytes >= L.split + L.split_bytes) {
    prm.split_ws = reinterpret_cast<float*>(w + L.split);
    split_cap = L.split_bytes;
  }
  int grid_ctas = 0;
  const int sa_ = epi.split_as;
  if constexpr (MODE == 6) {
    e = launch_leaf<MODE, 0, PAIR>(maps, prm, tiles, split_cap, sa_, s, &grid_ctas, hooks, cvp);
  } else {
    if (convert) {
      if constexpr (MODE == 3) e = launch_leaf<3, 0, true, true>(maps, prm, tiles, split_cap, sa_, s, &grid_ctas,
                                                                  hooks, cvp);
    } else if (epi.kind == 1) {
      e = launch_leaf<MODE, 1, PAIR>(maps, prm, tiles, split_cap, sa_, s, &grid_ctas, hooks, cvp);
    } else if (epi.kind == 2) {
      e = launch_leaf<MODE, 2, PAIR>(maps, prm, tiles, split_cap, sa_, s, &grid_ctas, hooks, cvp);
    } else {
      e = launch_leaf<MODE, 0, PAIR>(maps, prm, tiles, split_cap, sa_, s, &grid_ctas, hooks, cvp);
    }
  }
  if (e != cudaSuccess) return e;
  kernels += 1;
  if (rep) {
    rep->kernels = kernels;
    rep->grid_x = grid_ctas; rep->grid_y = 1; rep->grid_z = 1;
    rep->block_threads = THREADS;
    rep->tile_m = TM; rep->tile_n = C_::TN; rep->tile_k = C_::BK;
    rep->smem_bytes = (int)(C_::SMEM_BYTES + (convert ? CV_SMEM : 0));
    rep->literal = 0;
    rep->workspace_bytes = (int64_t)L.total;
  }
  return cudaSuccess;
}

int mode_of_tier(int tier) { return tier == 2 ? 3 : tier == 4 ? 8 : tier == 5 ? 6 : 1; }

// ---- batches of independent instances ----------------------------------------
template <int MODE>
cudaError_t launch_batch_kernels(const TcBatch& b, const DeviceStatus& st, cudaStream_t s,
                                 const LaunchHooks* hooks) {
  using C_ = Cfg<MODE>;
  constexpr int NPROD = MODE == 3 ? 3 : 1;
  ConvParams cvp{};
  if (b.convert) {
    // flags and claim counter zeroed, then the first round's blocks split
    // (marking their flags); the leaf's converters do the rest
    cudaError_t e = cudaMemsetAsync(b.d_flags, 0, b.flags_count * sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (b.num_pre_tiles > 0) {
      split_batch<NPROD><<<b.num_pre_tiles, 256, 0, s>>>(static_cast<const SplitOp*>(b.d_ops),
                                                         static_cast<const SplitTile*>(b.d_pre_tiles), b.d_flags);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    cvp.flags = b.d_flags;
    cvp.claim = b.d_flags + (b.flags_count - 4);
    cvp.chunks = static_cast<const SplitTile*>(b.d_chunks);
    cvp.ops = static_cast<const SplitOp*>(b.d_ops);
    cvp.num_chunks = b.num_chunks;
  } else if (b.num_split_tiles > 0) {
    split_batch<NPROD><<<b.num_split_tiles, 256, 0, s>>>(static_cast<const SplitOp*>(b.d_ops),
                                                         static_cast<const SplitTile*>(b.d_split_tiles), nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (b.num_tiles == 0) return cudaSuccess;
  alignas(64) CUtensorMap unused[6];
  memset(unused, 0, sizeof unused);
  TcParams prm{};
  prm.status = st.dev;
  prm.wait_limit_us = st.wait_limit_us;
  GroupParams gp{static_cast<const GroupInst*>(b.d_insts), static_cast<const GroupTile*>(b.d_tiles), b.num_tiles};
  if (b.tile_m > BM) {
    // 256-row tiles on CTA pairs: clusters of two
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b.grid);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = Cfg<MODE, true>::SMEM_BYTES + (b.convert ? CV_SMEM : 0);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    hook_begin(hooks, s);
    cudaError_t e;
    if constexpr (MODE == 3) {
      if (b.convert)
        e = cudaLaunchKernelEx(&cfg, sgemm_tc<3, 0, true, true, true>, unused[0], unused[1], unused[2], unused[3],
                               unused[4], unused[5], prm, gp, cvp);
      else
        e = cudaLaunchKernelEx(&cfg, sgemm_tc<3, 0, true, true, false>, unused[0], unused[1], unused[2], unused[3],
                               unused[4], unused[5], prm, gp, cvp);
    } else {
      e = cudaLaunchKernelEx(&cfg, sgemm_tc<MODE, 0, true, true, false>, unused[0], unused[1], unused[2],
                             unused[3], unused[4], unused[5], prm, gp, cvp);
    }
    hook_end(hooks, s);
    return e;
  }
  hook_begin(hooks, s);
  sgemm_tc<MODE, 0, true, false>
      <<<b.grid, THREADS, C_::SMEM_BYTES, s>>>(unused[0], unused[1], unused[2], unused[3], unused[4], unused[5], prm,
                                               gp, ConvParams{});
  hook_end(hooks, s);
  return cudaGetLastError();
}

void free_dev(void** p) {
  if (*p) cudaFree(*p);
  *p = nullptr;
}

template <class T>
int upload(void** dst, const std::vector<T>& v, std::string* err) {
  free_dev(dst);
  if (v.empty()) return 0;
  if (cudaMalloc(dst, v.size() * sizeof(T)) != cudaSuccess ||
      cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    *err = "cannot upload a batch table to the device";
    free_dev(dst);
    return -1;
  }
  return 0;
}

}  // namespace

int batch_tile_m(int policy) { return policy >= 4 ? 2 * BM : BM; }

std::vector<int> batch_choose_bn(const std::vector<SgemmDesc>& d, int policy) {
  std::vector<int> bn(d.size(), BN);
  const int rule = policy & 3, tm = batch_tile_m(policy);
  if (rule == 0) return bn;
  if (rule == 1) {
    std::fill(bn.begin(), bn.end(), 128);
    return bn;
  }
  // Model rules: for each instance pick the tile width that minimises
  // tiles x (columns x padded K + per-tile overhead), the overhead counted
  // in the same column-K units (rule 2: light, 3: heavy).
  const double overhead = rule == 2 ? 8192.0 : 65536.0;
  for (size_t i = 0; i < d.size(); ++i) {
    const double kp = (double)((d[i].K + 127) / 128 * 128);
    double best = -1;
    for (int w : {64, 128, 256}) {
      const double tiles = (double)((d[i].M + tm - 1) / tm) * (double)((d[i].N + w - 1) / w);
      const double cost = tiles * (w * kp + overhead);
      if (best < 0 || cost < best - 1e-9) {
        best = cost;
        bn[i] = w;
      }
    }
  }
  return bn;
}

int batch_schedule(const std::vector<SgemmDesc>& d, const std::vector<int>& bn, int units, std::vector<int>* tiles,
                   int tile_m) {
  // Every output tile (tile_m rows by its instance's width) of every
  // instance, longest first (cost: padded K x width x tile_m / 128 plus a
  // per-tile overhead), each given to the persistent unit (CTA, or CTA pair)
  // with the least work so far (LPT). Unit u runs slots u, u + G, u + 2G,
  // ...: slot r * G + u holds its r-th tile, or an empty record (instance
  // -1) when it has fewer tiles than the busiest unit. 4 ints per slot:
  // (instance, m0, n0, unit). Returns G, the units the launch needs.
  struct T {
    int64_t cost;
    int inst, m0, n0;
  };
  std::vector<T> v;
  for (size_t i = 0; i < d.size(); ++i) {
    if (d[i].M <= 0 || d[i].N <= 0) continue;
    const int64_t kp = (d[i].K + 127) / 128 * 128;
    for (int64_t n0 = 0; n0 < d[i].N; n0 += bn[i])
      for (int64_t m0 = 0; m0 < d[i].M; m0 += tile_m)
        v.push_back({kp * bn[i] * (tile_m / BM) + 4096, (int)i, (int)m0, (int)n0});
  }
  std::stable_sort(v.begin(), v.end(), [](const T& a, const T& b) { return a.cost > b.cost; });
  tiles->clear();
  if (v.empty()) return 1;
  const int G = std::max(1, std::min<int>((int)v.size(), units));
  std::vector<std::vector<int>> per(G);
  std::vector<int64_t> load(G, 0);
  // least loaded CTA, lowest index among equals (a linear scan: G <= a few hundred)
  for (size_t i = 0; i < v.size(); ++i) {
    int u = 0;
    for (int w = 1; w < G; ++w)
      if (load[w] < load[u]) u = w;
    per[u].push_back((int)i);
    load[u] += v[i].cost;
  }
  size_t rounds = 0;
  for (auto& q : per) rounds = std::max(rounds, q.size());
  for (size_t r = 0; r < rounds; ++r)
    for (int u = 0; u < G; ++u) {
      const bool has = r < per[u].size();
      const T& t = has ? v[per[u][r]] : v[0];
      tiles->push_back(has ? t.inst : -1);
      tiles->push_back(has ? t.m0 : 0);
      tiles->push_back(has ? t.n0 : 0);
      tiles->push_back(u);
    }
  return G;
}

// The grouped leaf's kernel attributes (dynamic shared memory, register
// split check) and how many persistent units it runs at once: one CTA per
// SM, or (PAIR) the clusters of two that fit, at most half the SMs.
template <int MODE, bool PAIR, bool CONVERT = false>
cudaError_t batch_kernel_setup(int* units) {
  using C_ = Cfg<MODE, PAIR>;
  auto kernel = sgemm_tc<MODE, 0, true, PAIR, CONVERT>;
  constexpr uint32_t smem = C_::SMEM_BYTES + (CONVERT ? CV_SMEM : 0);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = check_register_split(kernel);
  if (e != cudaSuccess) return e;
  if constexpr (!PAIR) {
    *units = num_sms();
  } else {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(2 * (num_sms() / 2));
    int n = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&n, kernel, &cfg)) != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    *units = std::min(n, num_sms() / 2);
  }
  return cudaSuccess;
}

int tc_batch_build(TcBatch* b, std::string* err) {
  const int mode = mode_of_tier(b->tier);
  const int count = (int)b->d.size();
  if (mode == 8) {
    *err = "batches run the BF16x3 and BF16 tiers";
    return -1;
  }
  // workspace: each instance's planes, 256-byte aligned, laid end to end
  if (!b->ws) {
    b->plane_off.assign(count, 0);
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
      b->plane_off[i] = off;
      off += ws_layout(b->d[i], mode).total;
      off = align256(off);
    }
    b->ws_bytes = std::max<size_t>(off, 256);
    if (cudaMalloc(&b->ws, b->ws_bytes) != cudaSuccess) {
      b->ws = nullptr;
      *err = "cannot allocate the batch's operand planes";
      return -1;
    }
    // split pre-pass tables (independent of the tile widths)
    std::vector<SplitOp> ops;
    std::vector<SplitTile> st;
    b->op_a.assign(count, -1);
    b->op_b.assign(count, -1);
    for (int i = 0; i < count; ++i) {
      const SgemmDesc& d = b->d[i];
      if (d.M <= 0 || d.N <= 0 || d.K <= 0) continue;
      b->op_a[i] = (int)ops.size();
      b->op_b[i] = (int)ops.size() + 1;
      const WsLayout L = ws_layout(d, mode);
      uint8_t* w = static_cast<uint8_t*>(b->ws) + b->plane_off[i];
      const SplitOp a{d.A, d.lda, d.transA ? 0 : 1, (int)d.M, (int)d.K, (int)L.Kp,
                      reinterpret_cast<__nv_bfloat16*>(w + L.a_hi), reinterpret_cast<__nv_bfloat16*>(w + L.a_lo)};
      const SplitOp bb{d.B, d.ldb, d.transB ? 1 : 0, (int)d.N, (int)d.K, (int)L.Kp,
                       reinterpret_cast<__nv_bfloat16*>(w + L.b_hi), reinterpret_cast<__nv_bfloat16*>(w + L.b_lo)};
      for (const SplitOp& o : {a, bb}) {
        const int id = (int)ops.size();
        ops.push_back(o);
        for (int r0 = 0; r0 < o.rows; r0 += 64)
          for (int k0 = 0; k0 < o.Kp; k0 += 64) st.push_back({id, r0, k0, -1});
      }
    }
    if (upload(&b->d_ops, ops, err) || upload(&b->d_split_tiles, st, err)) return -1;
    b->num_split_tiles = (int)st.size();
  }
  // kernel attributes first (so a run can be captured into a CUDA graph),
  // and the persistent units the leaf can run at once: CTAs, or CTA pairs
  const bool pair = b->policy >= 4;
  b->convert = b->policy >= 8;
  if (b->convert && mode != 3) {
    *err = "in-leaf conversion (policies 8-11) takes the BF16x3 tier";
    return -1;
  }
  int units = 0;
  cudaError_t e = mode == 3 ? (b->convert ? batch_kernel_setup<3, true, true>(&units)
                               : pair     ? batch_kernel_setup<3, true>(&units)
                                          : batch_kernel_setup<3, false>(&units))
                            : (pair ? batch_kernel_setup<1, true>(&units) : batch_kernel_setup<1, false>(&units));
  if (e != cudaSuccess) {
    *err = cudaGetErrorString(e);
    return -1;
  }
  // tile widths, tensor maps and the tile schedule of the current policy:
  // a CTA loads 128 rows of A and all bn rows of B of its tile; a pair's
  // CTAs 128 rows of A each and bn / 2 rows of B each
  b->bn = batch_choose_bn(b->d, b->policy);
  b->tile_m = batch_tile_m(b->policy);
  const int rb = pair ? (mode == 3 ? Cfg<3, true>::ROW_BYTES : Cfg<1, true>::ROW_BYTES)
                      : (mode == 3 ? Cfg<3>::ROW_BYTES : Cfg<1>::ROW_BYTES);
  std::vector<GroupInst> insts(count);
  for (int i = 0; i < count; ++i) {
    const SgemmDesc& d = b->d[i];
    GroupInst& g = insts[i];
    memset(&g, 0, sizeof g);
    g.C = d.C;
    g.ldc = d.ldc;
    g.M = (int)d.M;
    g.N = (int)d.N;
    g.K = (int)d.K;
    g.bn = b->bn[i];
    g.alpha = d.alpha;
    g.beta = d.beta;
    if (d.M <= 0 || d.N <= 0 || d.K <= 0) continue;
    const WsLayout L = ws_layout(d, mode);
    uint8_t* w = static_cast<uint8_t*>(b->ws) + b->plane_off[i];
    const int brows = pair ? g.bn / 2 : g.bn;
    if (!encode_plane(&g.tm[0], w + L.a_hi, (int)d.M, (int)d.K, (int)L.Kp, BM, 2, rb, err) ||
        !encode_plane(&g.tm[2], w + L.b_hi, (int)d.N, (int)d.K, (int)L.Kp, brows, 2, rb, err))
      return -1;
    if (mode == 3) {
      if (!encode_plane(&g.tm[1], w + L.a_lo, (int)d.M, (int)d.K, (int)L.Kp, BM, 2, rb, err) ||
          !encode_plane(&g.tm[3], w + L.b_lo, (int)d.N, (int)d.K, (int)L.Kp, brows, 2, rb, err))
        return -1;
    } else {
      g.tm[1] = g.tm[0];
      g.tm[3] = g.tm[2];
    }
  }
  std::vector<int> tiles;
  const int G = batch_schedule(b->d, b->bn, units, &tiles, b->tile_m);
  std::vector<GroupTile> gt(tiles.size() / 4);
  b->real_tiles = 0;
  for (size_t t = 0; t < gt.size(); ++t) {
    GroupTile& g = gt[t];
    memset(&g, 0, sizeof g);
    if (tiles[4 * t] < 0) continue;  // an empty slot: M = N = K = 0, nothing to do
    ++b->real_tiles;
    const GroupInst& in = insts[tiles[4 * t]];
    g.inst = tiles[4 * t];
    g.m0 = tiles[4 * t + 1];
    g.n0 = tiles[4 * t + 2];
    g.K = in.K;
    g.M = in.M;
    g.N = in.N;
    g.bn = in.bn;
    g.C = in.C;
    g.ldc = in.ldc;
    g.alpha = in.alpha;
    g.beta = in.beta;
  }
  if (b->convert) {
    // Flags: per instance, its A blocks' then its B blocks' (128 rows each),
    // a block's slabs (64 K each) padded to 4; the claim counter last.
    size_t off = 0;
    std::vector<int> kb4(count, 0);
    for (int i = 0; i < count; ++i) {
      const SgemmDesc& d = b->d[i];
      insts[i].flag_a = insts[i].flag_b = -1;
      if (b->op_a[i] < 0) continue;
      kb4[i] = (int)(((d.K + CV_BK - 1) / CV_BK + 3) / 4 * 4);
      insts[i].kb_stride = kb4[i];
      insts[i].flag_a = (int)off;
      off += (size_t)((d.M + CV_ROWS - 1) / CV_ROWS) * kb4[i];
      insts[i].flag_b = (int)off;
      off += (size_t)((d.N + CV_ROWS - 1) / CV_ROWS) * kb4[i];
    }
    if (off + 4 > (size_t)INT32_MAX) {
      *err = "too many conversion chunks for one batch";
      return -1;
    }
    b->flags_count = off + 4;  // (the counter at off, 16-byte padding)
    // Chunks in the order the schedule first reads them: round r = slots
    // [r G, (r + 1) G); the blocks round 0 reads are split before the launch
    // (64 x 64 tiles that mark their chunks' flags), those a later round
    // reads first are converted in the leaf, slab by slab across the round's
    // new blocks.
    struct Blk {
      int inst, op, blk;
    };
    std::vector<char> seen(off, 0);  // by a block's first flag
    std::vector<SplitTile> pre, chunks;
    const int slots = (int)(tiles.size() / 4);
    for (int r0 = 0; r0 < slots; r0 += G) {
      std::vector<Blk> fresh;
      for (int t = r0; t < std::min(slots, r0 + G); ++t) {
        const int i = tiles[4 * t];
        if (i < 0 || b->op_a[i] < 0) continue;
        const SgemmDesc& d = b->d[i];
        const int m0 = tiles[4 * t + 1], n0 = tiles[4 * t + 2], bn = b->bn[i];
        const int ablk = (int)((d.M + CV_ROWS - 1) / CV_ROWS), bblk = (int)((d.N + CV_ROWS - 1) / CV_ROWS);
        for (int q = m0 / CV_ROWS; q < std::min(ablk, (m0 + b->tile_m + CV_ROWS - 1) / CV_ROWS); ++q)
          fresh.push_back({i, 0, q});
        for (int q = n0 / CV_ROWS; q < std::min(bblk, (n0 + bn + CV_ROWS - 1) / CV_ROWS); ++q)
          fresh.push_back({i, 1, q});
      }
      std::vector<Blk> round;
      for (const Blk& x : fresh) {
        const int f = (x.op ? insts[x.inst].flag_b : insts[x.inst].flag_a) + x.blk * kb4[x.inst];
        if (seen[f]) continue;
        seen[f] = 1;
        round.push_back(x);
      }
      int max_kb = 0;
      for (const Blk& x : round) max_kb = std::max(max_kb, kb4[x.inst]);
      for (int kb = 0; kb < max_kb; ++kb) {
        for (const Blk& x : round) {
          const SgemmDesc& d = b->d[x.inst];
          const int nkb = (int)((d.K + CV_BK - 1) / CV_BK);
          if (kb >= nkb) continue;
          const int opi = x.op ? b->op_b[x.inst] : b->op_a[x.inst];
          const int f = (x.op ? insts[x.inst].flag_b : insts[x.inst].flag_a) + x.blk * kb4[x.inst] + kb;
          const int rows = (int)(x.op ? d.N : d.M);
          if (r0 == 0) {
            for (int rr = x.blk * CV_ROWS; rr < std::min(rows, (x.blk + 1) * CV_ROWS); rr += 64)
              pre.push_back({opi, rr, kb * CV_BK, f});
          } else {
            chunks.push_back({opi, x.blk * CV_ROWS, kb * CV_BK, f});
          }
        }
      }
    }
    free_dev(reinterpret_cast<void**>(&b->d_flags));
    if (cudaMalloc(reinterpret_cast<void**>(&b->d_flags), b->flags_count * sizeof(int)) != cudaSuccess) {
      b->d_flags = nullptr;
      *err = "cannot allocate the in-leaf conversion's flags";
      return -1;
    }
    if (upload(&b->d_chunks, chunks, err) || upload(&b->d_pre_tiles, pre, err)) return -1;
    b->num_chunks = (int)chunks.size();
    b->num_pre_tiles = (int)pre.size();
  }
  if (upload(&b->d_insts, insts, err) || upload(&b->d_tiles, gt, err)) return -1;
  b->num_tiles = (int)gt.size();
  b->grid = pair ? 2 * G : G;
  return 0;
}

cudaError_t tc_batch_run(const TcBatch& b, const DeviceStatus& st, cudaStream_t s, const LaunchHooks* hooks) {
  if (mode_of_tier(b.tier) == 3) return launch_batch_kernels<3>(b, st, s, hooks);
  return launch_batch_kernels<1>(b, st, s, hooks);
}

int tc_batch_autotune(TcBatch* b, const DeviceStatus& st, cudaStream_t s, int reps, int* best_policy,
                      double* best_ms, std::string* err) {
  int best = -1;
  double best_t = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // four width rules x single CTAs, CTA pairs, CTA pairs converting in the leaf (BF16x3)
  const int policies = mode_of_tier(b->tier) == 3 ? 12 : 8;
  for (int pol = 0; pol < policies; ++pol) {
    b->policy = pol;
    if (tc_batch_build(b, err)) break;
    if (tc_batch_run(*b, st, s, nullptr) != cudaSuccess) break;  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) tc_batch_run(*b, st, s, nullptr);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      *err = "a timed batch run failed";
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    const double t = ms / std::max(1, reps);
    if (best < 0 || t < best_t) {
      best = pol;
      best_t = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0) {
    if (err->empty()) *err = "autotuning failed";
    return -1;
  }
  b->policy = best;
  if (tc_batch_build(b, err)) return -1;
  *best_policy = best;
  *best_ms = best_t;
  return 0;
}

cudaError_t launch_wait_selftest(const DeviceStatus& st, uint64_t limit_ns, cudaStream_t s) {
  wait_selftest<<<1, 32, 0, s>>>(st.dev, limit_ns);
  return cudaGetLastError();
}

void tc_batch_free(TcBatch* b) {
  free_dev(reinterpret_cast<void**>(&b->d_flags));
  free_dev(&b->d_chunks);
  free_dev(&b->d_pre_tiles);
  free_dev(&b->ws);
  free_dev(&b->d_ops);
  free_dev(&b->d_split_tiles);
  free_dev(&b->d_insts);
  free_dev(&b->d_tiles);
}

namespace {

}  // namespace

void tc_tile(int tier, int* tm, int* tn) {
  const int mode = mode_of_tier(tier);
  *tm = pair_for_mode(mode) ? 2 * BM : BM;  // a CTA pair's tile, or one CTA's
  *tn = Cfg<1>::TN;
  (void)mode;
}

size_t tc_workspace_bytes(const SgemmDesc& d, int tier) { return ws_layout(d, mode_of_tier(tier)).total; }

int tc_num_sms() { return num_sms(); }

cudaError_t launch_tc(const SgemmDesc& d, int tier, void* ws, size_t ws_bytes, const DeviceStatus& st,
                      cudaStream_t s, KernelReport* rep, std::string* err, const LaunchHooks* hooks,
                      const Epilogue& epi, const OperandPlanes& pa, const OperandPlanes& pb) {
  if (d.M > INT32_MAX / 2 || d.N > INT32_MAX / 2 || d.K > INT32_MAX / 2) {
    *err = "M, N and K must each fit in 30 bits for the tensor-core tiers";
    return cudaErrorInvalidValue;
  }
  // the planes are required; the tail split's region is used when present
  if (ws_bytes < ws_layout(d, mode_of_tier(tier)).planes || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0) {
    *err = "workspace too small or not 256-byte aligned";
    return cudaErrorInvalidValue;
  }
  if (tier == 2) return run_tc<3>(d, ws, ws_bytes, st, s, rep, err, hooks, epi, pa, pb);
  if (tier == 4) return run_tc<8>(d, ws, ws_bytes, st, s, rep, err, hooks, epi, pa, pb);
  if (tier == 5) return run_tc<6>(d, ws, ws_bytes, st, s, rep, err, hooks, epi, pa, pb);
  return run_tc<1>(d, ws, ws_bytes, st, s, rep, err, hooks, epi, pa, pb);
}

OperandLayout tc_operand_layout(int tier, int64_t rows, int64_t K) {
  return operand_layout(rows, K, mode_of_tier(tier));
}

}  // namespace hpvm

// ===========================================================================
// Allocation-free BF16x3 leaf (hpvm_sgemm_bf16x3_noalloc).
//
// Some callers cannot allocate device memory when they call the leaf: code
// that runs inside another framework's memory pool (which has reserved the
// device memory and forbids its plugins to call cudaMalloc), code on a
// latency-critical thread (cudaMalloc and cudaFree may synchronise the
// device), or code that must not fail for lack of memory halfway through a
// job. For them this entry point keeps the split BF16 planes in a fixed
// file-scope device array instead of a workspace. The array is allocated
// when the library's kernels are loaded onto a GPU and stays allocated on
// every GPU that loads the library until the process exits.
namespace hpvm {
namespace {

constexpr size_t kNoAllocScratchBytes = HPVM_NOALLOC_SCRATCH_BYTES;

// The scratch planes. Host code must not use this name as a device address;
// it gets the address through cudaGetSymbolAddress (see noalloc_scratch).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// The calling thread's current CUDA context (the driver's cuCtxGetCurrent,
// reached through the runtime's entry-point query), or null.
CUcontext current_context() {
  using Fn = CUresult (*)(CUcontext*);
  static Fn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<Fn>(f);
  });
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Device address of g_noalloc_scratch on the current device, looked up with
// that device current and cached per device together with the context it
// belongs to. A device reset (cudaDeviceReset) gives the device a new
// context, in which the array has a new address: the lookup is then made
// again. Returns nullptr and a message on failure.
void* noalloc_scratch(std::string* err) {
  static std::mutex mu;
  static void* addr[kMaxDevices] = {nullptr};
  static CUcontext owner[kMaxDevices] = {nullptr};
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *err = "no usable current CUDA device";
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  const CUcontext ctx = current_context();
  if (!addr[dev] || !ctx || ctx != owner[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      addr[dev] = nullptr;
      *err = std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e);
      return nullptr;
    }
    addr[dev] = p;
    owner[dev] = current_context();  // the lookup made the device's context current if it was not
  }
  return addr[dev];
}

}  // namespace
}  // namespace hpvm

extern "C" int hpvm_sgemm_bf16x3_noalloc(int64_t M, int64_t N, int64_t K, float alpha, const float* A,
                                         int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                                         int64_t ldc, int transA, int transB, int* dev_status,
                                         void* cuda_stream) {
  using namespace hpvm;
  if (M < 0 || N < 0 || K < 0) return set_last_error(HPVM_ERR_SHAPE, "negative M, N or K");
  const int64_t ar = transA ? K : M, br = transB ? N : K;
  if (lda < std::max<int64_t>(1, ar) || ldb < std::max<int64_t>(1, br) || ldc < std::max<int64_t>(1, M))
    return set_last_error(HPVM_ERR_SHAPE, "a leading dimension is smaller than the rows of its matrix");
  if (M == 0 || N == 0) return set_last_error(HPVM_OK, "");
  if (!C || (K > 0 && (!A || !B))) return set_last_error(HPVM_ERR_INVALID_ARG, "A, B or C is NULL");
  SgemmDesc d;
  d.M = M;
  d.N = N;
  d.K = K;
  d.A = A;
  d.lda = lda;
  d.B = B;
  d.ldb = ldb;
  d.C = C;
  d.ldc = ldc;
  d.alpha = alpha;
  d.beta = beta;
  d.transA = transA != 0;
  d.transB = transB != 0;
  // the planes must fit; the tail split runs when the rest of the array
  // also holds its partial sums, else the leaf runs whole tiles only
  const size_t need = ws_layout(d, 3).planes;
  if (need > kNoAllocScratchBytes || M > INT32_MAX / 2 || N > INT32_MAX / 2 || K > INT32_MAX / 2) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "the split planes need %zu bytes, more than the %zu-byte scratch array of the "
             "allocation-free entry point: use hpvm_launch with a workspace",
             need, kNoAllocScratchBytes);
    return set_last_error(HPVM_ERR_SHAPE, buf);
  }
  std::string err;
  void* ws = noalloc_scratch(&err);
  if (!ws) return set_last_error(HPVM_ERR_CUDA, err.c_str());
  DeviceStatus st;
  st.dev = dev_status;
  cudaError_t e = launch_tc(d, 2, ws, kNoAllocScratchBytes, st, static_cast<cudaStream_t>(cuda_stream),
                            nullptr, &err, nullptr);
  if (e == cudaErrorInvalidValue && !err.empty()) return set_last_error(HPVM_ERR_SHAPE, err.c_str());
  if (e != cudaSuccess) return set_last_error(HPVM_ERR_CUDA, cudaGetErrorString(e));
  return set_last_error(HPVM_OK, "");
}

// ===========================================================================
// Operand preparation of the tensor-core tiers, callable on its own.
extern "C" int hpvm_split_bf16(const float* X, int64_t ld, int kcontig, int64_t rows, int64_t K, void* hi,
                               void* lo, void* cuda_stream) {
  using namespace hpvm;
  if (rows < 0 || K < 0 || rows > INT32_MAX / 2 || K > INT32_MAX / 2)
    return set_last_error(HPVM_ERR_SHAPE, "rows and K must be in [0, 2^30)");
  if (rows == 0 || K == 0) return set_last_error(HPVM_OK, "");
  if (!X || !hi) return set_last_error(HPVM_ERR_INVALID_ARG, "X or hi is NULL");
  if (ld < (kcontig ? K : rows)) return set_last_error(HPVM_ERR_SHAPE, "ld is smaller than the contiguous extent");
  if ((reinterpret_cast<uintptr_t>(hi) & 15u) || (reinterpret_cast<uintptr_t>(lo) & 15u))
    return set_last_error(HPVM_ERR_ALIGN, "hi and lo must be 16-byte aligned");
  const int Kp = (int)((K + 7) / 8 * 8);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = lo ? launch_split<3>(X, ld, !kcontig, (int)rows, (int)K, Kp, static_cast<__nv_bfloat16*>(hi),
                                       static_cast<__nv_bfloat16*>(lo), nullptr, s)
                     : launch_split<1>(X, ld, !kcontig, (int)rows, (int)K, Kp, static_cast<__nv_bfloat16*>(hi),
                                       nullptr, nullptr, s);
  if (e != cudaSuccess) return set_last_error(HPVM_ERR_CUDA, cudaGetErrorString(e));
  return set_last_error(HPVM_OK, "");
}

extern "C" int hpvm_split3_bf16(const float* X, int64_t ld, int kcontig, int64_t rows, int64_t K, void* hi,
                                void* mid, void* lo, void* cuda_stream) {
  using namespace hpvm;
  if (rows < 0 || K < 0 || rows > INT32_MAX / 2 || K > INT32_MAX / 2)
    return set_last_error(HPVM_ERR_SHAPE, "rows and K must be in [0, 2^30)");
  if (rows == 0 || K == 0) return set_last_error(HPVM_OK, "");
  if (!X || !hi || !mid || !lo) return set_last_error(HPVM_ERR_INVALID_ARG, "X, hi, mid or lo is NULL");
  if (ld < (kcontig ? K : rows)) return set_last_error(HPVM_ERR_SHAPE, "ld is smaller than the contiguous extent");
  if ((reinterpret_cast<uintptr_t>(hi) | reinterpret_cast<uintptr_t>(mid) | reinterpret_cast<uintptr_t>(lo)) & 15u)
    return set_last_error(HPVM_ERR_ALIGN, "hi, mid and lo must be 16-byte aligned");
  const int Kp = (int)((K + 7) / 8 * 8);
  cudaError_t e = launch_split<6>(X, ld, !kcontig, (int)rows, (int)K, Kp, static_cast<__nv_bfloat16*>(hi),
                                  static_cast<__nv_bfloat16*>(mid), static_cast<__nv_bfloat16*>(lo),
                                  static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return set_last_error(HPVM_ERR_CUDA, cudaGetErrorString(e));
  return set_last_error(HPVM_OK, "");
}

extern "C" int hpvm_quant_fp8(const float* X, int64_t ld, int kcontig, int64_t rows, int64_t K, void* q,
                              float* scales, void* cuda_stream) {
  using namespace hpvm;
  if (rows < 0 || K < 0 || rows > INT32_MAX / 2 || K > INT32_MAX / 2)
    return set_last_error(HPVM_ERR_SHAPE, "rows and K must be in [0, 2^30)");
  if (rows == 0 || K == 0) return set_last_error(HPVM_OK, "");
  if (!X || !q || !scales) return set_last_error(HPVM_ERR_INVALID_ARG, "X, q or scales is NULL");
  if (ld < (kcontig ? K : rows)) return set_last_error(HPVM_ERR_SHAPE, "ld is smaller than the contiguous extent");
  if (reinterpret_cast<uintptr_t>(q) & 15u) return set_last_error(HPVM_ERR_ALIGN, "q must be 16-byte aligned");
  const int Kp = (int)((K + 15) / 16 * 16);
  const int nkb = (int)((K + FP8_BLOCK - 1) / FP8_BLOCK);
  cudaError_t e = launch_quant(X, ld, !kcontig, (int)rows, (int)K, Kp, static_cast<uint8_t*>(q), scales, nkb,
                               static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return set_last_error(HPVM_ERR_CUDA, cudaGetErrorString(e));
  return set_last_error(HPVM_OK, "");
}
