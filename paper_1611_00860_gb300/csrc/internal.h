// Internal interface between the graph runtime (runtime.cpp) and the kernel
// launchers (fp32_leaf.cu, tc_leaf.cu). Not part of the C-ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace hpvm {

// One lowered sgemm leaf: C <- alpha*op(A)*op(B) + beta*C, column-major.
struct SgemmDesc {
  int64_t M = 0, N = 0, K = 0;
  const float* A = nullptr;
  int64_t lda = 1;
  const float* B = nullptr;
  int64_t ldb = 1;
  float* C = nullptr;
  int64_t ldc = 1;
  float alpha = 1.f, beta = 0.f;
  int transA = 0, transB = 0;
};

// What a launcher ran (copied into hpvm_launch_info).
struct KernelReport {
  int kernels = 0;
  int grid_x = 0, grid_y = 0, grid_z = 0;
  int block_threads = 0;
  int tile_m = 0, tile_n = 0, tile_k = 0;
  int smem_bytes = 0;
  int literal = 0;
  int64_t workspace_bytes = 0;
};

// Status word the tensor-core kernels write when a bounded wait expires.
// Bits: which wait gave up (see tc_leaf.cu).
struct DeviceStatus {
  int* dev = nullptr;   // device-visible address (mapped pinned memory)
  int* host = nullptr;  // host address of the same word
  uint32_t wait_limit_us = 0;  // limit of each bounded wait in the kernels (0: 2 s)
};

// Optional CUDA events recorded on the launch stream right before and right
// after the main (leaf) kernel of a launch, for timing that kernel alone.
struct LaunchHooks {
  cudaEvent_t main_begin = nullptr;
  cudaEvent_t main_end = nullptr;
};
inline void hook_begin(const LaunchHooks* h, cudaStream_t s) {
  if (h && h->main_begin) cudaEventRecord(h->main_begin, s);
}
inline void hook_end(const LaunchHooks* h, cudaStream_t s) {
  if (h && h->main_end) cudaEventRecord(h->main_end, s);
}

// Elementwise leaf merged into (or run after) a sgemm leaf:
// kind 1: C <- tanh(C); kind 2: C <- C * (1 - H^2) with H column-major (ldaux).
// fwd (tensor-core BF16x3 and BF16 leaves only): the epilogue also writes
// the operand planes of its result for a later leaf that reads this C as
// op(B) = B with K = this M (a streaming edge between stages): column n of
// C becomes plane row n, at the offsets tc_operand_layout(tier, N, M) gives
// from fwd. Those planes equal what that leaf's own conversion of C makes.
// rows (same tiers): the epilogue also writes the planes of C with rows of
// C as operand rows (row m of C is plane row m, K = N) at the offsets
// tc_operand_layout(tier, M, N) gives from rows: the planes a later leaf
// reading C as op(A) = A or op(B) = B^T converts from C, bit for bit.
// split_as (>= 0): the leaf splits its last round's tiles only where the
// leaf with that merged elementwise kind would, so an unmerged stage (a
// plain leaf, then the elementwise kernel) rounds as the merged one does.
struct Epilogue {
  int kind = 0;
  const float* aux = nullptr;
  int64_t ldaux = 0;
  void* fwd = nullptr;
  void* rows = nullptr;
  int split_as = -1;
  bool planes_only = false;  // store the planes above only, not C itself
  // run the operand split as its own kernels even where the BF16x3 leaf
  // would write the planes itself (the same planes, bit for bit)
  bool separate_split = false;
};
// Standalone elementwise kernel on the M x N column-major C (fp32_leaf.cu).
cudaError_t launch_elementwise(const SgemmDesc& d, const Epilogue& e, cudaStream_t s);

// ---- FP32 CUDA-core leaves (fp32_leaf.cu) ---------------------------------
// Literal Section 3.4 mapping: CTA (bx, by) = internal instance, thread
// (tx, ty) = leaf instance, tiles of the Allocation node in shared memory.
cudaError_t launch_fp32_dfg(const SgemmDesc& d, int block, int grid_x,
                            int grid_y, size_t tile_bytes, cudaStream_t s,
                            KernelReport* rep, const LaunchHooks* hooks);
// Register-tiled FP32 kernel.
cudaError_t launch_fp32_tiled(const SgemmDesc& d, cudaStream_t s,
                              KernelReport* rep, const LaunchHooks* hooks);
void fp32_tiled_tile(int* tm, int* tn);

// ---- tensor-core leaves (tc_leaf.cu) --------------------------------------
// tier: 2 = BF16x3 split, 3 = BF16, 4 = FP8, 5 = BF16x6 split (plain
// epilogue only). `epi` is fused into the leaf's epilogue (after
// alpha*acc + beta*C).
size_t tc_workspace_bytes(const SgemmDesc& d, int tier);
// Returns a cudaError_t; on a host-side precondition failure returns
// cudaErrorInvalidValue and fills *err.
// Planes of one operand kept outside the workspace (the context's plane
// cache): `base` holds the hi plane, the lo plane (BF16x3) and the block
// scales (FP8) at the offsets tc_operand_layout gives. ready: they already
// hold the operand, so its conversion is skipped; otherwise it is converted
// into them and `converted` (if set) is recorded on the stream right after.
struct OperandPlanes {
  void* base = nullptr;
  bool ready = false;
  cudaEvent_t converted = nullptr;
};
struct OperandLayout {
  size_t hi = 0, lo = 0, scales = 0, total = 0;
  size_t lo2 = 0;  // BF16x6: the third part's plane
};
OperandLayout tc_operand_layout(int tier, int64_t rows, int64_t K);
cudaError_t launch_tc(const SgemmDesc& d, int tier, void* ws, size_t ws_bytes,
                      const DeviceStatus& st, cudaStream_t s,
                      KernelReport* rep, std::string* err,
                      const LaunchHooks* hooks, const Epilogue& epi = Epilogue(),
                      const OperandPlanes& pa = OperandPlanes(), const OperandPlanes& pb = OperandPlanes());
void tc_tile(int tier, int* tm, int* tn);

// ---- batches of independent instances (tc_leaf.cu) ------------------------
// One batch of sgemm instances run by the grouped persistent leaf: the split
// pre-pass of every operand in one launch, then every output tile of every
// instance in one launch (tiles in decreasing cost, round robin over CTAs).
struct TcBatch {
  int tier = 2;
  std::vector<SgemmDesc> d;
  std::vector<int> bn;  // tile width of each instance (the policy's choice)
  // width rule (policy & 3): 0: 256, 1: 128, 2/3: cost model (light/heavy
  // tile overhead); policy 0-3 on single CTAs (128-row tiles), 4-7 on CTA
  // pairs (256-row tiles), 8-11 on CTA pairs converting the operands in the
  // leaf (BF16x3)
  int policy = 2;
  int tile_m = 128;     // rows of an output tile (the policy's height)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  std::vector<size_t> plane_off;
  void* d_ops = nullptr;
  void* d_split_tiles = nullptr;
  int num_split_tiles = 0;
  void* d_insts = nullptr;
  void* d_tiles = nullptr;
  int num_tiles = 0;   // slots of the schedule (output tiles and empty slots)
  int real_tiles = 0;  // output tiles
  int grid = 0;
  // in-leaf conversion (policies 8-11, BF16x3): the operand records of each
  // instance (index into the split's operand table, -1 for none), the
  // flags (and claim counter) region, the chunk list the leaf's converters
  // claim from, and the first round's split tiles
  std::vector<int> op_a, op_b;
  bool convert = false;
  int* d_flags = nullptr;
  size_t flags_count = 0;  // ints, the claim counter last
  void* d_chunks = nullptr;
  int num_chunks = 0;
  void* d_pre_tiles = nullptr;
  int num_pre_tiles = 0;
};
std::vector<int> batch_choose_bn(const std::vector<SgemmDesc>& d, int policy);
// rows of a batch tile under a policy: 128 (single CTAs) or 256 (CTA pairs)
int batch_tile_m(int policy);
// tiles: 4 ints per slot (instance, m0, n0, unit) in schedule order
int batch_schedule(const std::vector<SgemmDesc>& d, const std::vector<int>& bn, int units, std::vector<int>* tiles,
                   int tile_m);
// SMs of the current device (148 when none answers): the persistent CTAs a
// batch's leaf launch uses.
int tc_num_sms();
int tc_batch_build(TcBatch* b, std::string* err);
cudaError_t tc_batch_run(const TcBatch& b, const DeviceStatus& st, cudaStream_t s, const LaunchHooks* hooks);
int tc_batch_autotune(TcBatch* b, const DeviceStatus& st, cudaStream_t s, int reps, int* best_policy,
                      double* best_ms, std::string* err);
void tc_batch_free(TcBatch* b);
// One kernel whose single bounded wait can never be satisfied (tc_leaf.cu).
cudaError_t launch_wait_selftest(const DeviceStatus& st, uint64_t limit_ns, cudaStream_t s);

// Sets the calling thread's hpvm_last_error() message (cleared for HPVM_OK)
// and returns `code` (runtime.cpp).
int set_last_error(int code, const char* msg);

}  // namespace hpvm
