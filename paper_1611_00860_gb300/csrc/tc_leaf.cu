// Tensor-core (tcgen05) lowerings of the SgemmLeaf node (Section 5.1) for
// sm_103a: the BF16x3 split tier and the plain BF16 tier.
//
// The leaf computes C <- alpha*op(A)*op(B) + beta*C (column-major FP32, C
// not read when beta == 0). The paper computes in FP32 on CUDA cores; here
// each FP32 operand x is split into BF16 parts hi = bf16_rn(x) and
// lo = bf16_rn(x - hi) and the leaf sums the three products
// hi*hi + hi*lo + lo*hi on the tensor cores into one FP32 accumulator in
// tensor memory (the BF16 tier keeps hi*hi only).
//
// Mapping of the dataflow graph (Section 4.4): one internal-node instance
// (an output tile of BM x BN) is one CTA; the Allocation node's tile memory
// is a ring of STAGES shared-memory slabs filled by TMA (the paper's scratch-
// pad tiles), plus the accumulator tile in tensor memory; the replicated
// leaf's multiply-accumulate is a sequence of tcgen05.mma instructions.
//
// Kernels
//   split_mmajor / split_kmajor: FP32 op(X) -> K-major BF16 hi (and lo)
//       planes in the workspace, rows of Kp = roundup(K, 8) elements.
//   sgemm_tc<NPROD>: warp 0 issues TMA loads, warp 1 allocates tensor
//       memory and issues the MMAs, warps 2..5 read the accumulator
//       (tcgen05.ld) and write C. Every mbarrier wait is bounded; on
//       expiry the kernel sets a bit in the status word, drains its own
//       copies and MMAs (bounded again), frees tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
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
constexpr int BK = 32;              // K slab in BF16 elements = 64 bytes
constexpr int MMA_K = 16;           // K per tcgen05.mma kind::f16
constexpr int EPI_WARPS = 8;        // two per tensor-memory lane quarter
constexpr int THREADS = 64 + EPI_WARPS * 32;  // producer, MMA, epilogue warps
constexpr uint32_t TMEM_COLS = 2 * BN;        // two FP32 BM x BN chunk buffers
constexpr int KC_SLABS = 4;         // K chunk = 4 slabs = 128 elements; its
                                    // sum is added to FP32 registers with
                                    // round-to-nearest (the tensor-core
                                    // accumulation truncates)
constexpr int GROUP_N = 8;          // column tiles per rasterisation group
constexpr uint32_t A_SLAB = BM * BK * 2;  // bytes of one A plane slab
constexpr uint32_t B_SLAB = BN * BK * 2;  // bytes of one B plane slab
constexpr uint32_t SMEM_BUDGET = 200 * 1024;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s per bounded wait

// status bits (DeviceStatus word)
constexpr int ST_PRODUCER = 1, ST_MMA = 2, ST_EPILOGUE = 4, ST_DRAIN = 8;

template <int NPROD>
struct Cfg {
  static constexpr int PLANES = NPROD == 3 ? 2 : 1;
  static constexpr uint32_t STAGE_BYTES = PLANES * (A_SLAB + B_SLAB);
  static constexpr int STAGES = (int)((SMEM_BUDGET - 2048) / STAGE_BYTES) > 8
                                    ? 8 : (int)((SMEM_BUDGET - 2048) / STAGE_BYTES);
  static constexpr uint32_t SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 512 /*barriers*/;
  static_assert(2 * STAGES * 8 + 4 * 8 + 8 <= 512, "barrier area");
};

struct TcParams {
  int M, N, K;
  float* C;
  int64_t ldc;
  float alpha, beta;
  int* status;
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
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `bar` with the given parity. Gives up (returns
// false) when another role raised the abort flag or after WAIT_LIMIT_NS, in
// which case it records `code` in the status word and raises the flag.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int* status, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t n = 1;; ++n) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((n & 63u) == 0) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > WAIT_LIMIT_NS) {
        if (status) atomicOr_system(status, code);
        *abort_flag = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint64_t* bar, void* dst, int c0,
                                            int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of tcgen05 (K-major, 64-byte swizzle):
// start address >> 4 in bits 0-13, leading byte offset >> 4 in 16-29 (not
// used by swizzled K-major layouts), stride byte offset >> 4 in 32-45 (the
// distance between groups of 8 rows: 8 * 64 bytes), descriptor version 1 in
// bits 46-47, swizzle mode in bits 61-63 (4 = 64-byte swizzle).
__device__ __forceinline__ uint64_t sdesc_k_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>(512 >> 4) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(4) << 61;
  return d;
}
// Instruction descriptor of tcgen05.mma kind::f16: D format F32 (bits 4-5 =
// 1), A and B BF16 (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
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

// ---- operand split ------------------------------------------------------------
__device__ __forceinline__ void split_pair(float x, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(x);
  l = __float2bfloat16_rn(x - __bfloat162float(h));
}

// X "m-major": element (r, k) at X[r + k*ld] (rows contiguous). 64 x 64 tiles.
template <int NPROD>
__global__ void __launch_bounds__(256) split_mmajor(const float* __restrict__ X, int64_t ld, int rows, int K,
                                                    int Kp, __nv_bfloat16* __restrict__ hi,
                                                    __nv_bfloat16* __restrict__ lo) {
  __shared__ float t[64][65];
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * 64, k0 = (int64_t)blockIdx.y * 64;
#pragma unroll 4
  for (int it = 0; it < 16; ++it) {
    int e = tid + it * 256;
    int kk = e >> 6, rr = e & 63;
    int64_t gr = r0 + rr, gk = k0 + kk;
    t[kk][rr] = (gr < rows && gk < K) ? X[gr + gk * ld] : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    int e = tid + it * 256;
    int rr = e >> 3, kc = (e & 7) * 8;
    int64_t gr = r0 + rr, gk = k0 + kc;
    if (gr >= rows || gk >= Kp) continue;
    __align__(16) __nv_bfloat16 h[8];
    __align__(16) __nv_bfloat16 l[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) split_pair(t[kc + u][rr], h[u], l[u]);
    *reinterpret_cast<uint4*>(hi + gr * Kp + gk) = *reinterpret_cast<const uint4*>(h);
    if (NPROD == 3) *reinterpret_cast<uint4*>(lo + gr * Kp + gk) = *reinterpret_cast<const uint4*>(l);
  }
}

// X "k-major": element (r, k) at X[k + r*ld] (K contiguous).
template <int NPROD>
__global__ void __launch_bounds__(256) split_kmajor(const float* __restrict__ X, int64_t ld, int rows, int K,
                                                    int Kp, __nv_bfloat16* __restrict__ hi,
                                                    __nv_bfloat16* __restrict__ lo) {
  const int64_t chunks = Kp / 8;
  const int64_t total = (int64_t)rows * chunks;
  for (int64_t task = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; task < total;
       task += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = task / chunks, k = (task % chunks) * 8;
    const float* src = X + r * ld + k;
    __align__(16) __nv_bfloat16 h[8];
    __align__(16) __nv_bfloat16 l[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) split_pair((k + u < K) ? src[u] : 0.f, h[u], l[u]);
    *reinterpret_cast<uint4*>(hi + r * Kp + k) = *reinterpret_cast<const uint4*>(h);
    if (NPROD == 3) *reinterpret_cast<uint4*>(lo + r * Kp + k) = *reinterpret_cast<const uint4*>(l);
  }
}

// ---- the leaf kernel -------------------------------------------------------------
// Persistent: CTA b handles tiles b, b + gridDim.x, ... in a grouped order
// (GROUP_N column tiles at a time, M fastest) so CTAs that run together share
// operand panels in L2.
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int* m0, int* n0) {
  const int group = GROUP_N * tiles_m;
  const int g = t / group, r = t % group;
  const int first_n = g * GROUP_N;
  const int gn = min(GROUP_N, tiles_n - first_n);
  *m0 = (r / gn) * BM;
  *n0 = (first_n + r % gn) * BN;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int NPROD>
__global__ void __launch_bounds__(THREADS, 1)
    sgemm_tc(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
             const __grid_constant__ CUtensorMap tmB_hi, const __grid_constant__ CUtensorMap tmB_lo,
             TcParams p) {
  using C_ = Cfg<NPROD>;
  constexpr int S = C_::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * C_::STAGE_BYTES);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;   // [2] MMA -> epilogue: chunk accumulated in buffer b
  uint64_t* tempty = tfull + 2;  // [2] epilogue -> MMA: buffer b read out
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int num_kb = (p.K + BK - 1) / BK;
  const int num_chunks = (num_kb + KC_SLABS - 1) / KC_SLABS;
  const int tiles_m = (p.M + BM - 1) / BM, tiles_n = (p.N + BN - 1) / BN;
  const int num_tiles = tiles_m * tiles_n;

  // stage s: [A hi][A lo][B hi][B lo] (lo planes only for NPROD == 3)
  auto a_hi = [&](int s) { return smem + s * C_::STAGE_BYTES; };
  auto a_lo = [&](int s) { return smem + s * C_::STAGE_BYTES + A_SLAB; };
  auto b_hi = [&](int s) { return smem + s * C_::STAGE_BYTES + C_::PLANES * A_SLAB; };
  auto b_lo = [&](int s) { return smem + s * C_::STAGE_BYTES + C_::PLANES * A_SLAB + B_SLAB; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EPI_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // bookkeeping for the drain after an abort
  int issued = 0;     // producer: slabs requested (ring position)
  int committed = 0;  // MMA: slabs whose MMAs were committed (ring position)
  int chunks_committed = 0;

  if (warp == 0 && lane == 0) {
    // ---- producer: TMA loads of the operand slabs into the ring
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA_hi)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB_hi)) : "memory");
    int it = 0;
    bool go = true;
    for (int t = blockIdx.x; go && t < num_tiles; t += gridDim.x) {
      int m0, n0;
      tile_coords(t, tiles_m, tiles_n, &m0, &n0);
      for (int kb = 0; kb < num_kb; ++kb, ++it) {
        const int s = it % S;
        const uint32_t ph = (it / S) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1, abort_flag, p.status, ST_PRODUCER)) {
          go = false;
          break;
        }
        mbar_expect_tx(&full[s], C_::STAGE_BYTES);
        const int k = kb * BK;
        tma_load_2d(&tmA_hi, &full[s], a_hi(s), k, m0);
        if (NPROD == 3) tma_load_2d(&tmA_lo, &full[s], a_lo(s), k, m0);
        tma_load_2d(&tmB_hi, &full[s], b_hi(s), k, n0);
        if (NPROD == 3) tma_load_2d(&tmB_lo, &full[s], b_lo(s), k, n0);
        issued = it + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: per K chunk, a fresh accumulation in tensor-memory
    // buffer (chunk parity); three (or one) BF16 products per 16-wide K step
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    int it = 0, g = 0;
    bool go = true;
    for (int t = blockIdx.x; go && t < num_tiles; t += gridDim.x) {
      for (int c = 0; go && c < num_chunks; ++c, ++g) {
        const int buf = g & 1;
        const uint32_t use = (uint32_t)(g >> 1);
        if (!mbar_wait(&tempty[buf], (use & 1) ^ 1, abort_flag, p.status, ST_MMA)) {
          go = false;
          break;
        }
        tc_fence_after();
        const uint32_t dst = tmem + buf * BN;
        const int kb_end = min(num_kb, (c + 1) * KC_SLABS);
        for (int kb = c * KC_SLABS; kb < kb_end; ++kb, ++it) {
          const int s = it % S;
          const uint32_t ph = (it / S) & 1;
          if (!mbar_wait(&full[s], ph, abort_flag, p.status, ST_MMA)) {
            go = false;
            break;
          }
          tc_fence_after();
          const uint32_t ah = smem_u32(a_hi(s)), al = smem_u32(a_lo(s));
          const uint32_t bh = smem_u32(b_hi(s)), bl = smem_u32(b_lo(s));
#pragma unroll
          for (int kk = 0; kk < BK / MMA_K; ++kk) {
            const uint32_t off = kk * MMA_K * 2;  // bytes along the 64-byte row
            const uint32_t acc = (kb == c * KC_SLABS && kk == 0) ? 0u : 1u;
            if (NPROD == 3) {
              umma_bf16(dst, sdesc_k_sw64(al + off), sdesc_k_sw64(bh + off), idesc, acc);
              umma_bf16(dst, sdesc_k_sw64(ah + off), sdesc_k_sw64(bl + off), idesc, 1u);
              umma_bf16(dst, sdesc_k_sw64(ah + off), sdesc_k_sw64(bh + off), idesc, 1u);
            } else {
              umma_bf16(dst, sdesc_k_sw64(ah + off), sdesc_k_sw64(bh + off), idesc, acc);
            }
          }
          umma_commit(&empty[s]);  // frees the slab once these MMAs have read it
          committed = it + 1;
        }
        if (!go) break;
        umma_commit(&tfull[buf]);  // chunk complete in buffer buf
        chunks_committed = g + 1;
      }
    }
  } else if (warp >= 2) {
    // ---- epilogue: every chunk, tensor memory -> FP32 registers (round to
    // nearest); at the end of a tile, registers -> C, coalesced per column
    const int q = warp & 3;          // TMEM lane quarter this warp may access
    const int h = (warp - 2) >> 2;   // which half of the BN columns
    int g = 0;
    bool go = true;
    for (int t = blockIdx.x; go && t < num_tiles; t += gridDim.x) {
      int m0, n0;
      tile_coords(t, tiles_m, tiles_n, &m0, &n0);
      float acc[BN / 2];
#pragma unroll
      for (int u = 0; u < BN / 2; ++u) acc[u] = 0.f;
      for (int c = 0; c < num_chunks; ++c, ++g) {
        const int buf = g & 1;
        const uint32_t use = (uint32_t)(g >> 1);
        if (!mbar_wait(&tfull[buf], use & 1, abort_flag, p.status, ST_EPILOGUE)) {
          go = false;
          break;
        }
        tc_fence_after();
        __syncwarp();
        const uint32_t src = tmem + (static_cast<uint32_t>(q * 32) << 16) + buf * BN + h * (BN / 2);
#pragma unroll
        for (int i = 0; i < BN / 64; ++i) {
          uint32_t r[32];
          tmem_ld_x32(src + i * 32, r);
#pragma unroll
          for (int u = 0; u < 32; ++u) acc[i * 32 + u] += __uint_as_float(r[u]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[buf]);
      }
      if (!go) break;
      const int row = m0 + q * 32 + lane;
      const int col0 = n0 + h * (BN / 2);
      if (row < p.M) {
        float* cp = p.C + row + (int64_t)col0 * p.ldc;
#pragma unroll
        for (int u = 0; u < BN / 2; ++u) {
          if (col0 + u < p.N) {
            float* e = cp + (int64_t)u * p.ldc;
            *e = (p.beta == 0.f) ? p.alpha * acc[u] : fmaf(p.alpha, acc[u], p.beta * *e);
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    // Drain what this CTA itself started before returning (bounded waits):
    // TMA loads not yet consumed, and the MMAs of the last commit.
    if (warp == 0 && lane == 0) {
      for (int it = (issued > S ? issued - S : 0); it < issued; ++it) {
        const int s = it % S;
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&full[s], (it / S) & 1)) {
          if (globaltimer() - t0 > WAIT_LIMIT_NS) {
            if (p.status) atomicOr_system(p.status, ST_DRAIN);
            break;
          }
        }
      }
    }
    if (warp == 1 && lane == 0 && committed > 0) {
      const int it = committed - 1;
      const int s = it % S;
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&empty[s], (it / S) & 1)) {
        if (globaltimer() - t0 > WAIT_LIMIT_NS) {
          if (p.status) atomicOr_system(p.status, ST_DRAIN);
          break;
        }
      }
    }
    (void)chunks_committed;
    __syncthreads();
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
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

// K-major BF16 plane: rows x K elements, row stride Kp elements; box BK x box_rows.
bool encode_plane(CUtensorMap* map, const void* base, int rows, int K, int Kp, int box_rows,
                  std::string* err) {
  auto enc = get_encoder();
  if (!enc) {
    *err = "cuTensorMapEncodeTiled is not available from the driver";
    return false;
  }
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[160];
    snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d) for a %d x %d plane", (int)r, rows, K);
    *err = buf;
    return false;
  }
  return true;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
  }
  return n;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
inline int64_t kpad(int64_t K) { return (K + 7) / 8 * 8; }

template <int NPROD>
cudaError_t launch_split(const float* X, int64_t ld, bool mmajor, int rows, int K, int Kp,
                         __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t s) {
  if (rows == 0 || K == 0) return cudaSuccess;
  if (mmajor) {
    dim3 grid((rows + 63) / 64, (Kp + 63) / 64);
    split_mmajor<NPROD><<<grid, 256, 0, s>>>(X, ld, rows, K, Kp, hi, lo);
  } else {
    int64_t tasks = (int64_t)rows * (Kp / 8);
    int64_t blocks = (tasks + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    split_kmajor<NPROD><<<(unsigned)blocks, 256, 0, s>>>(X, ld, rows, K, Kp, hi, lo);
  }
  return cudaGetLastError();
}

template <int NPROD>
cudaError_t run_tc(const SgemmDesc& d, void* ws, const DeviceStatus& st, cudaStream_t s, KernelReport* rep,
                   std::string* err, const LaunchHooks* hooks) {
  using C_ = Cfg<NPROD>;
  const int M = (int)d.M, N = (int)d.N, K = (int)d.K;
  const int Kp = (int)kpad(K);
  uint8_t* w = static_cast<uint8_t*>(ws);
  const size_t a_plane = align256((size_t)M * Kp * 2), b_plane = align256((size_t)N * Kp * 2);
  __nv_bfloat16* ah = reinterpret_cast<__nv_bfloat16*>(w);
  __nv_bfloat16* al = reinterpret_cast<__nv_bfloat16*>(w + a_plane);
  __nv_bfloat16* bh = reinterpret_cast<__nv_bfloat16*>(w + C_::PLANES * a_plane);
  __nv_bfloat16* bl = reinterpret_cast<__nv_bfloat16*>(w + C_::PLANES * a_plane + b_plane);
  int kernels = 0;
  cudaError_t e;
  if (K > 0) {
    // op(A) rows are contiguous when A is not transposed; op(B)'s N rows when B is
    e = launch_split<NPROD>(d.A, d.lda, !d.transA, M, K, Kp, ah, al, s);
    if (e != cudaSuccess) return e;
    e = launch_split<NPROD>(d.B, d.ldb, d.transB != 0, N, K, Kp, bh, bl, s);
    if (e != cudaSuccess) return e;
    kernels += 2;
  }
  alignas(64) CUtensorMap maps[4];
  memset(maps, 0, sizeof maps);
  if (K > 0) {
    if (!encode_plane(&maps[0], ah, M, K, Kp, BM, err) || !encode_plane(&maps[2], bh, N, K, Kp, BN, err))
      return cudaErrorInvalidValue;
    if (NPROD == 3) {
      if (!encode_plane(&maps[1], al, M, K, Kp, BM, err) || !encode_plane(&maps[3], bl, N, K, Kp, BN, err))
        return cudaErrorInvalidValue;
    } else {
      maps[1] = maps[0];
      maps[3] = maps[2];
    }
  }
  static bool attr_set = false;
  if (!attr_set) {
    e = cudaFuncSetAttribute(sgemm_tc<NPROD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C_::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  TcParams prm{M, N, K, d.C, d.ldc, d.alpha, d.beta, st.dev};
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  dim3 grid((unsigned)std::min(tiles, num_sms()));
  hook_begin(hooks, s);
  sgemm_tc<NPROD><<<grid, THREADS, C_::SMEM_BYTES, s>>>(maps[0], maps[1], maps[2], maps[3], prm);
  hook_end(hooks, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  kernels += 1;
  if (rep) {
    rep->kernels = kernels;
    rep->grid_x = (int)grid.x; rep->grid_y = (int)grid.y; rep->grid_z = 1;
    rep->block_threads = THREADS;
    rep->tile_m = BM; rep->tile_n = BN; rep->tile_k = BK;
    rep->smem_bytes = (int)C_::SMEM_BYTES;
    rep->literal = 0;
    rep->workspace_bytes = (int64_t)(C_::PLANES * (a_plane + b_plane));
  }
  return cudaSuccess;
}

}  // namespace

void tc_tile(int /*tier*/, int* tm, int* tn) {
  *tm = BM;
  *tn = BN;
}

size_t tc_workspace_bytes(const SgemmDesc& d, int tier) {
  const int planes = tier == 2 ? 2 : 1;
  const int64_t Kp = kpad(d.K);
  return planes * (align256((size_t)d.M * Kp * 2) + align256((size_t)d.N * Kp * 2));
}

cudaError_t launch_tc(const SgemmDesc& d, int tier, void* ws, size_t ws_bytes, const DeviceStatus& st,
                      cudaStream_t s, KernelReport* rep, std::string* err, const LaunchHooks* hooks) {
  if (d.M > INT32_MAX / 2 || d.N > INT32_MAX / 2 || d.K > INT32_MAX / 2) {
    *err = "M, N and K must each fit in 30 bits for the tensor-core tiers";
    return cudaErrorInvalidValue;
  }
  if (ws_bytes < tc_workspace_bytes(d, tier) || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0) {
    *err = "workspace too small or not 256-byte aligned";
    return cudaErrorInvalidValue;
  }
  if (tier == 2) return run_tc<3>(d, ws, st, s, rep, err, hooks);
  return run_tc<1>(d, ws, st, s, rep, err, hooks);
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

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (with that device current) and cached. Returns nullptr and a
// message on failure.
void* noalloc_scratch(std::string* err) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static void* addr[kMaxDevices] = {nullptr};
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *err = "no usable current CUDA device";
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      *err = std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e);
      return nullptr;
    }
    addr[dev] = p;
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
  const size_t need = tc_workspace_bytes(d, 2);
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
