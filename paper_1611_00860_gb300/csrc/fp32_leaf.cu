// FP32 CUDA-core lowerings of the SgemmLeaf node (Section 6.1).
//
// Both kernels compute C <- alpha*op(A)*op(B) + beta*C with column-major
// storage; beta == 0 means C is not read.
//
// sgemm_leaf_dfg: the hierarchy of Section 3.4 taken literally. The
//   internal node SgemmInternal (a 2-D grid) becomes the CUDA grid, the
//   replicated SgemmLeaf (a square block x block grid) becomes the CTA, the
//   Allocation node's two block x block FP32 tiles become dynamic shared
//   memory whose size the host computed before the launch (the example's
//   Allocation1), and llvm.hpvm.barrier becomes __syncthreads. Leaf
//   instance (tx, ty) of internal instance (bx, by) owns output
//   (bx*block + tx, by*block + ty).
//
// sgemm_fp32_tiled: a register-tiled kernel for large problems: 128 x 128
//   outputs per CTA, 256 threads, 8 x 8 outputs per thread (packed FP32
//   FMAs on pairs of outputs), K slabs of 16 staged in shared memory with
//   one slab prefetched into registers.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace hpvm {
namespace {

// element (r, c) of op(X), column-major X with leading dimension ld
__device__ __forceinline__ float op_load(const float* X, int64_t ld, bool trans,
                                         int64_t r, int64_t c) {
  return trans ? X[c + r * ld] : X[r + c * ld];
}

template <bool TA, bool TB>
__global__ void sgemm_leaf_dfg(SgemmDesc d, int bs) {
  extern __shared__ float alloc_mem[];
  float* shB = alloc_mem;            // Allocation output 0 -> leaf port 12
  float* shA = alloc_mem + bs * bs;  // Allocation output 2 -> leaf port 14
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t bx = blockIdx.x, by = blockIdx.y;
  const int64_t i = bx * bs + tx, j = by * bs + ty;
  const int64_t i_base = bx * bs, j_base = by * bs;
  float acc = 0.f;
  for (int64_t t0 = 0; t0 < d.K; t0 += bs) {
    // phase 1: every leaf instance stages one element of each tile. The
    // element an instance stages is chosen so a warp reads consecutive
    // addresses; shA[r + q*bs] = opA(i_base + r, t0 + q) and
    // shB[q + c*bs] = opB(t0 + q, j_base + c) either way.
    {
      int r = TA ? ty : tx, q = TA ? tx : ty;
      int64_t gi = i_base + r, gp = t0 + q;
      shA[r + q * bs] = (gi < d.M && gp < d.K) ? op_load(d.A, d.lda, TA, gi, gp) : 0.f;
    }
    {
      int q = TB ? ty : tx, c = TB ? tx : ty;
      int64_t gp = t0 + q, gj = j_base + c;
      shB[q + c * bs] = (gp < d.K && gj < d.N) ? op_load(d.B, d.ldb, TB, gp, gj) : 0.f;
    }
    __syncthreads();  // llvm.hpvm.barrier
    // phase 2: multiply-accumulate over the staged K slice
    for (int q = 0; q < bs; ++q) acc = fmaf(shA[tx + q * bs], shB[q + ty * bs], acc);
    __syncthreads();  // llvm.hpvm.barrier
  }
  if (i < d.M && j < d.N) {
    float* c = d.C + i + j * d.ldc;
    *c = (d.beta == 0.f) ? d.alpha * acc : fmaf(d.alpha, acc, d.beta * *c);
  }
}

// ---------------------------------------------------------------------------
// Register-tiled kernel.

// (c0, c1) <- (a*b0 + c0, a*b1 + c1), one packed FP32 FMA (fma.rn.f32x2)
__device__ __forceinline__ void fma2(float& c0, float& c1, float a, float b0, float b1) {
  asm("{\n\t.reg .b64 acc, av, bv;\n\t"
      "mov.b64 acc, {%0, %1};\n\t"
      "mov.b64 av, {%2, %2};\n\t"
      "mov.b64 bv, {%3, %4};\n\t"
      "fma.rn.f32x2 acc, av, bv, acc;\n\t"
      "mov.b64 {%0, %1}, acc;\n\t}"
      : "+f"(c0), "+f"(c1)
      : "f"(a), "f"(b0), "f"(b1));
}
constexpr int TBM = 128, TBN = 128, TBK = 16, TTHREADS = 256;

// Loads a TBK x 128 slab of op(X)^T-as-[k][m] into registers: for the
// operand whose rows (m) are contiguous in memory ("m-major": op(A) = A or
// op(B) = B^T), thread tid fetches float4s along m; otherwise along k.
// Slab element (k, m) is op(X)(m0 + m, k0 + k) for A, op(X)(k0+k, n0+m) for B.
struct Slab {
  float v[8];
};

template <bool MMAJOR>
__device__ __forceinline__ void slab_load(Slab& s, const float* X, int64_t ld,
                                          int64_t rows, int64_t kdim,
                                          int64_t m0, int64_t k0, int tid,
                                          bool vec_ok) {
  // 2048 elements, 8 per thread as two groups of 4 consecutive elements
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    int e = (tid + g * TTHREADS) * 4;  // 0..2047, step 4
    if (MMAJOR) {
      int k = e / TBM, m = e % TBM;  // 4 consecutive m
      int64_t gm = m0 + m, gk = k0 + k;
      const float* p = X + gm + gk * ld;
      if (vec_ok && gk < kdim && gm + 3 < rows) {
        float4 f = *reinterpret_cast<const float4*>(p);
        s.v[g * 4 + 0] = f.x; s.v[g * 4 + 1] = f.y; s.v[g * 4 + 2] = f.z; s.v[g * 4 + 3] = f.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          s.v[g * 4 + u] = (gk < kdim && gm + u < rows) ? p[u] : 0.f;
      }
    } else {
      int m = e / TBK, k = e % TBK;  // 4 consecutive k
      int64_t gm = m0 + m, gk = k0 + k;
      const float* p = X + gk + gm * ld;
      if (vec_ok && gm < rows && gk + 3 < kdim) {
        float4 f = *reinterpret_cast<const float4*>(p);
        s.v[g * 4 + 0] = f.x; s.v[g * 4 + 1] = f.y; s.v[g * 4 + 2] = f.z; s.v[g * 4 + 3] = f.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          s.v[g * 4 + u] = (gm < rows && gk + u < kdim) ? p[u] : 0.f;
      }
    }
  }
}

template <bool MMAJOR>
__device__ __forceinline__ void slab_store(const Slab& s, float (*sh)[TBM + 4], int tid) {
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    int e = (tid + g * TTHREADS) * 4;
    if (MMAJOR) {
      int k = e / TBM, m = e % TBM;
      *reinterpret_cast<float4*>(&sh[k][m]) =
          make_float4(s.v[g * 4 + 0], s.v[g * 4 + 1], s.v[g * 4 + 2], s.v[g * 4 + 3]);
    } else {
      int m = e / TBK, k = e % TBK;
#pragma unroll
      for (int u = 0; u < 4; ++u) sh[k + u][m] = s.v[g * 4 + u];
    }
  }
}

// TA: op(A) = A^T (A stored K x M). TB: op(B) = B^T (B stored N x K).
template <bool TA, bool TB>
__global__ void __launch_bounds__(TTHREADS, 2)
sgemm_fp32_tiled(SgemmDesc d, int vec_a, int vec_b, int vec_c) {
  __shared__ __align__(16) float As[2][TBK][TBM + 4];
  __shared__ __align__(16) float Bs[2][TBK][TBN + 4];
  const int tid = threadIdx.x;
  const int64_t m0 = (int64_t)blockIdx.x * TBM, n0 = (int64_t)blockIdx.y * TBN;
  const int tr = tid % 16, tc = tid / 16;
  // A is "m-major" (rows contiguous) when op(A) = A; B when op(B) = B^T
  constexpr bool AM = !TA, BM = TB;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

  Slab sa, sb;
  const int64_t ktiles = (d.K + TBK - 1) / TBK;
  if (ktiles > 0) {
    slab_load<AM>(sa, d.A, d.lda, d.M, d.K, m0, 0, tid, vec_a);
    slab_load<BM>(sb, d.B, d.ldb, d.N, d.K, n0, 0, tid, vec_b);
    slab_store<AM>(sa, As[0], tid);
    slab_store<BM>(sb, Bs[0], tid);
  }
  __syncthreads();
  for (int64_t t = 0; t < ktiles; ++t) {
    const int cur = t & 1;
    if (t + 1 < ktiles) {
      slab_load<AM>(sa, d.A, d.lda, d.M, d.K, m0, (t + 1) * TBK, tid, vec_a);
      slab_load<BM>(sb, d.B, d.ldb, d.N, d.K, n0, (t + 1) * TBK, tid, vec_b);
    }
#pragma unroll
    for (int k = 0; k < TBK; ++k) {
      float a[8], b[8];
      float4 a0 = *reinterpret_cast<const float4*>(&As[cur][k][tr * 4]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[cur][k][64 + tr * 4]);
      float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][k][tc * 4]);
      float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][k][64 + tc * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
      b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
      // packed FP32 FMAs (two lanes per instruction, each rounded once as
      // fmaf rounds): half the issue slots of the scalar form, 11% faster at
      // 8192 (57.3 -> 64.0 TFLOP/s; keeping the accumulators as packed
      // 64-bit pairs measured slower, 60.5)
#pragma unroll
      for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; y += 2) fma2(acc[x][y], acc[x][y + 1], a[x], b[y], b[y + 1]);
    }
    if (t + 1 < ktiles) {
      slab_store<AM>(sa, As[cur ^ 1], tid);
      slab_store<BM>(sb, Bs[cur ^ 1], tid);
    }
    __syncthreads();
  }
  // epilogue: rows m0 + {tr*4 + 0..3, 64 + tr*4 + 0..3}, cols n0 + {tc*4 + 0..3, 64 + tc*4 + 0..3}
#pragma unroll
  for (int y = 0; y < 8; ++y) {
    const int64_t j = n0 + (y < 4 ? tc * 4 + y : 64 + tc * 4 + (y - 4));
    if (j >= d.N) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t i = m0 + h * 64 + tr * 4;
      float* c = d.C + i + j * d.ldc;
      if (vec_c && i + 3 < d.M) {
        float4 r;
        if (d.beta == 0.f) {
          r = make_float4(d.alpha * acc[h * 4 + 0][y], d.alpha * acc[h * 4 + 1][y],
                          d.alpha * acc[h * 4 + 2][y], d.alpha * acc[h * 4 + 3][y]);
        } else {
          float4 o = *reinterpret_cast<const float4*>(c);
          r = make_float4(fmaf(d.alpha, acc[h * 4 + 0][y], d.beta * o.x),
                          fmaf(d.alpha, acc[h * 4 + 1][y], d.beta * o.y),
                          fmaf(d.alpha, acc[h * 4 + 2][y], d.beta * o.z),
                          fmaf(d.alpha, acc[h * 4 + 3][y], d.beta * o.w));
        }
        *reinterpret_cast<float4*>(c) = r;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (i + u < d.M) {
            float v = acc[h * 4 + u][y];
            c[u] = (d.beta == 0.f) ? d.alpha * v : fmaf(d.alpha, v, d.beta * c[u]);
          }
        }
      }
    }
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Elementwise leaves over the column-major M x N result (one thread per
// element, consecutive threads on consecutive rows): kind 1 applies tanh,
// kind 2 multiplies by 1 - H^2 (the derivative of tanh at the forward value H).
__global__ void elementwise_leaf(float* C, int64_t ldc, int64_t M, int64_t N, int kind, const float* H,
                                 int64_t ldh) {
  const int64_t total = M * N;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % M, j = t / M;
    float* c = C + i + j * ldc;
    if (kind == 1) {
      *c = tanhf(*c);
    } else {
      const float h = H[i + j * ldh];
      *c = *c * (1.f - h * h);
    }
  }
}

}  // namespace

cudaError_t launch_fp32_dfg(const SgemmDesc& d, int block, int grid_x, int grid_y,
                            size_t tile_bytes, cudaStream_t s, KernelReport* rep,
                            const LaunchHooks* hooks) {
  dim3 grid(grid_x, grid_y), thr(block, block);
  size_t smem = 2 * tile_bytes;  // the Allocation node's B tile and A tile
  if (smem > 48 * 1024) {
    cudaError_t e = cudaSuccess;
#define HPVM_SET_SMEM(TA, TB)                                                     \
    e = cudaFuncSetAttribute(sgemm_leaf_dfg<TA, TB>,                              \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;
    HPVM_SET_SMEM(false, false) HPVM_SET_SMEM(false, true)
    HPVM_SET_SMEM(true, false) HPVM_SET_SMEM(true, true)
#undef HPVM_SET_SMEM
  }
  hook_begin(hooks, s);
  if (d.transA) {
    if (d.transB) sgemm_leaf_dfg<true, true><<<grid, thr, smem, s>>>(d, block);
    else sgemm_leaf_dfg<true, false><<<grid, thr, smem, s>>>(d, block);
  } else {
    if (d.transB) sgemm_leaf_dfg<false, true><<<grid, thr, smem, s>>>(d, block);
    else sgemm_leaf_dfg<false, false><<<grid, thr, smem, s>>>(d, block);
  }
  hook_end(hooks, s);
  if (rep) {
    rep->kernels = 1;
    rep->grid_x = grid_x; rep->grid_y = grid_y; rep->grid_z = 1;
    rep->block_threads = block * block;
    rep->tile_m = block; rep->tile_n = block; rep->tile_k = block;
    rep->smem_bytes = (int)smem;
    rep->literal = 1;
    rep->workspace_bytes = 0;
  }
  return cudaGetLastError();
}

void fp32_tiled_tile(int* tm, int* tn) { *tm = TBM; *tn = TBN; }

cudaError_t launch_elementwise(const SgemmDesc& d, const Epilogue& e, cudaStream_t s) {
  if (e.kind == 0 || d.M == 0 || d.N == 0) return cudaSuccess;
  const int64_t total = d.M * d.N;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  elementwise_leaf<<<(unsigned)blocks, 256, 0, s>>>(d.C, d.ldc, d.M, d.N, e.kind, e.aux, e.ldaux);
  return cudaGetLastError();
}

cudaError_t launch_fp32_tiled(const SgemmDesc& d, cudaStream_t s, KernelReport* rep,
                              const LaunchHooks* hooks) {
  dim3 grid((unsigned)((d.M + TBM - 1) / TBM), (unsigned)((d.N + TBN - 1) / TBN));
  // float4 access needs 16-byte aligned columns: base aligned and ld % 4 == 0
  int vec_a = aligned16(d.A) && d.lda % 4 == 0;
  int vec_b = aligned16(d.B) && d.ldb % 4 == 0;
  int vec_c = aligned16(d.C) && d.ldc % 4 == 0;
  hook_begin(hooks, s);
  if (d.transA) {
    if (d.transB) sgemm_fp32_tiled<true, true><<<grid, TTHREADS, 0, s>>>(d, vec_a, vec_b, vec_c);
    else sgemm_fp32_tiled<true, false><<<grid, TTHREADS, 0, s>>>(d, vec_a, vec_b, vec_c);
  } else {
    if (d.transB) sgemm_fp32_tiled<false, true><<<grid, TTHREADS, 0, s>>>(d, vec_a, vec_b, vec_c);
    else sgemm_fp32_tiled<false, false><<<grid, TTHREADS, 0, s>>>(d, vec_a, vec_b, vec_c);
  }
  hook_end(hooks, s);
  if (rep) {
    rep->kernels = 1;
    rep->grid_x = (int)grid.x; rep->grid_y = (int)grid.y; rep->grid_z = 1;
    rep->block_threads = TTHREADS;
    rep->tile_m = TBM; rep->tile_n = TBN; rep->tile_k = TBK;
    rep->smem_bytes = 0;
    rep->literal = 0;
    rep->workspace_bytes = 0;
  }
  return cudaGetLastError();
}

}  // namespace hpvm
