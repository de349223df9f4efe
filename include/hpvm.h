/*
 * hpvm.h -- C-ABI of the GB300 runtime for HPVM hierarchical dataflow graphs
 * (Kotsifakou et al., "HPVM: A Portable Virtual Instruction Set for
 * Heterogeneous Parallel Systems", arXiv 1611.00860).
 *
 * The calls mirror the paper's intrinsics (Table 1 and the intrinsic list of
 * Section 2.2): a program builds a hierarchical dataflow graph (DFG) of
 * internal nodes (which only hold child graphs), allocation leaves and
 * compute leaves, connects them with ordinary edges, binds parent inputs to
 * child inputs, then launches the graph on a CUDA stream and waits for it.
 * The runtime lowers the one graph shape it supports -- the sgemm example of
 * Section 6.1 -- onto hand-written sm_103a kernels.
 *
 * Conventions shared by every call
 *   - Every function returns HPVM_OK (0) or a negative HPVM_ERR_* code and
 *     never aborts. On error, hpvm_last_error() returns a message for the
 *     calling thread; nothing the call would have created is created.
 *   - Handles (hpvm_ctx, hpvm_node, hpvm_edge, hpvm_graph) are opaque. Nodes
 *     and edges belong to the context that created them and are freed by
 *     hpvm_cleanup(). A graph handle returned by hpvm_launch() is freed by a
 *     hpvm_wait() that returns HPVM_OK or an error other than HPVM_ERR_TIMEOUT.
 *   - Pointers inside argument records are device pointers (CUDA device or
 *     managed memory), or host pointers previously registered with
 *     hpvm_track_mem(). They are borrowed: the caller keeps them alive and
 *     leaves them untouched from hpvm_launch() until hpvm_wait() returns.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef HPVM_GB300_HPVM_H
#define HPVM_GB300_HPVM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HPVM_API __attribute__((visibility("default")))
#else
#define HPVM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------- */
#define HPVM_OK 0
#define HPVM_ERR_INVALID_ARG (-1)   /* null handle, bad enum, bad port number */
#define HPVM_ERR_INVALID_GRAPH (-2) /* breaks a rule of Section 2.1/2.2 */
#define HPVM_ERR_UNSUPPORTED (-3)   /* valid graph the runtime cannot lower */
#define HPVM_ERR_SHAPE (-4)         /* ld < rows, buffer bytes too small, ... */
#define HPVM_ERR_ALIGN (-5)         /* operand alignment a kernel needs */
#define HPVM_ERR_CUDA (-6)          /* a CUDA runtime/driver call failed */
#define HPVM_ERR_TIMEOUT (-7)       /* hpvm_wait ran out of time */
#define HPVM_ERR_DEVICE_FAULT (-8)  /* a kernel reported a bounded wait expired */
#define HPVM_ERR_NO_DEVICE (-9)     /* call needs a device; context is host-only */
#define HPVM_ERR_OUT_OF_MEMORY (-10)

/* ---- node kinds: the node function a node runs ------------------------ */
#define HPVM_NODE_INTERNAL 0   /* graph intrinsics only (Section 2.2) */
#define HPVM_NODE_ALLOCATION 1 /* allocation leaf (Section 3.4): tile memory */
#define HPVM_NODE_SGEMM_LEAF 2 /* the SgemmLeaf node function (Section 6.1);
                                  outputs 0, 1: its result C and bytesC */
/* Elementwise leaves over a column-major M x N matrix, updated in place;
 * outputs 0, 1: the matrix and its bytes. Joined to a SgemmLeaf of the same
 * grid by one-to-one edges (SgemmLeaf out 0 -> in 0, out 1 -> in 1) they are
 * merged into it (MergeDependentNodes, Section 4.1).
 * TANH_LEAF inputs: 0 X, 1 bytesX, 2 ldx, 3 M, 4 N; X <- tanh(X).
 * TANH_GRAD_LEAF inputs: 0 G, 1 bytesG, 2 ldg, 3 M, 4 N, 5 H, 6 bytesH,
 * 7 ldh; G <- G * (1 - H^2) (the adjoint of tanh at the output H). */
#define HPVM_NODE_TANH_LEAF 3
#define HPVM_NODE_TANH_GRAD_LEAF 4

/* ---- edge replication (Section 2.1) ----------------------------------- */
#define HPVM_ONE_TO_ONE 0 /* instance i -> instance i; grids must match */
#define HPVM_ALL_TO_ALL 1 /* every source instance -> every sink instance */

/* ---- leaf precision tiers (how the runtime lowers the SgemmLeaf) ------
 * FP32_DFG: one CUDA thread per leaf instance, one CTA per internal
 *           instance, the Allocation node's tiles in shared memory (the
 *           mapping of Section 3.4 taken literally); FP32 FMA.
 * FP32:     register-tiled FP32 CUDA-core kernel (same result definition).
 * BF16X3:   tcgen05 tensor cores, each FP32 operand split into BF16
 *           hi + lo, three products hi*hi + hi*lo + lo*hi, FP32 accumulate.
 * BF16:     tcgen05 tensor cores, operands rounded to BF16, FP32 accumulate.
 * BF16X6:   tcgen05 tensor cores, each FP32 operand split into three BF16
 *           parts hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid)
 *           (hi + mid + lo == x for every x of normal FP32 range, beyond
 *           2^-110 or so in magnitude), six products lo*hi + hi*lo + mid*mid
 *           + mid*hi + hi*mid + hi*hi (the three dropped ones are below 2^-25
 *           of hi*hi), FP32 accumulate. Twice the tensor work of BF16X3, for
 *           inputs on which two BF16 parts are not enough: a result dominated
 *           by a few rows and columns of large magnitude (say log-normal row
 *           scales) inherits the 2^-17 relative error of the two-part split
 *           in its few dominant elements, and BF16X3 can then miss 5e-6
 *           normwise even in exact arithmetic. Plain epilogue only: a merged
 *           elementwise leaf runs as its own kernel, and the plane cache
 *           flags CACHE_C / PLANES_ONLY and forwarded planes do not apply.
 * FP8:      tcgen05 kind::f8f6f4, op(A) and op(B) quantised to E4M3 with one
 *           FP32 scale per 128 x 128 block (scale = amax/448, round to
 *           nearest even, saturating); each 128-wide K block's product is
 *           scaled by its two block scales and summed in FP32 registers.
 */
#define HPVM_TIER_FP32_DFG 0
#define HPVM_TIER_FP32 1
#define HPVM_TIER_BF16X3 2
#define HPVM_TIER_BF16 3
#define HPVM_TIER_FP8 4
#define HPVM_TIER_BF16X6 5

/* A replication extent that is not a constant but the value of input port p
 * of the parent node at run time (the example passes its own block_x,
 * block_y, grid_x, grid_y arguments to createNode2D, Section 6.1). */
#define HPVM_DIM_FROM_INPUT(p) (-1 - (int64_t)(p))

/* launch flags (hpvm_sgemm_root_args.flags) */
#define HPVM_LAUNCH_NO_EVENT 1 /* no completion event: hpvm_wait syncs the
                                  stream (use inside CUDA graph capture) */
#define HPVM_LAUNCH_NO_FUSION 2 /* run a dependent elementwise leaf as its own
                                   kernel instead of merging it */
/* Operand plane cache (tensor tiers; no counterpart in the paper). The
 * BF16x3, BF16 and FP8 leaves read op(A) and op(B) as K-major BF16 / E4M3
 * planes converted from the FP32 operands. With these flags a stage keeps
 * the planes of an operand in its context, keyed by (device pointer, leading
 * dimension, rows, K, layout, tier), so that later launches can skip the
 * conversion:
 *   CACHE: convert op(X) into the cache (replacing what an entry with the
 *          same key held) and keep it;
 *   REUSE: the caller guarantees op(X) holds the values it held when its
 *          planes were cached: use them (converting and caching if the
 *          cache has none). Reusing planes of an operand that changed
 *          gives the product of the old values.
 * Launches on other streams that read or refill an entry are ordered by
 * CUDA events. The cache grows up to 4 GiB; beyond that operands are
 * converted into the workspace as without the flags. hpvm_drop_planes
 * frees it.
 * CACHE_C: a stage whose epilogue applies a merged elementwise leaf (BF16
 *          or BF16x3 tier, fusion on) also writes the planes of its result
 *          C, read with C's rows as operand rows, into the cache: the entry
 *          a later launch finds with REUSE_A for op(A) = A over C (lda =
 *          ldc, M = C's rows, K = C's columns) or REUSE_B for op(B) = B^T
 *          over C, the same planes that launch would convert from C, bit
 *          for bit. Other stages drop what such an entry holds, so a later
 *          REUSE converts. */
#define HPVM_LAUNCH_CACHE_A 4
#define HPVM_LAUNCH_REUSE_A 8
#define HPVM_LAUNCH_CACHE_B 16
#define HPVM_LAUNCH_REUSE_B 32
#define HPVM_LAUNCH_CACHE_C 64
/* PLANES_ONLY (tensor tiers, fusion on, beta = 0): the caller reads this
 * stage's result only through the planes the launch writes of it: the B
 * planes a streaming edge forwards to the next stage, and with CACHE_C the
 * cached row planes. The FP32 C is then not stored (it keeps its old
 * contents), saving its write. Ignored, and C stored, where those planes are
 * not all written (no forwarding and no CACHE_C entry, a CACHE_C entry the
 * cache had no room for, beta != 0, an unmerged stage, FP8, or C in a
 * tracked host region). A later launch that converts C instead of reusing
 * the planes (hpvm_drop_planes in between, or no REUSE flag) reads the old
 * contents. */
#define HPVM_LAUNCH_PLANES_ONLY 128
/* SEPARATE_SPLIT: the plain BF16X3 leaf normally converts most of its
 * operands itself when both have their rows contiguous (op(A) = A, op(B) =
 * B^T, the example's form), 16-byte aligned with leading dimensions that
 * are multiples of 4, and the first round of 256 x 256 tiles reads at most
 * half of their rows (large launches, e.g. 8192^3): the split kernels then
 * convert only the first round's rows, and the leaf's two otherwise idle
 * control warps convert the rest chunk by chunk while the leaf runs, each
 * slab's loads waiting for its chunks (the planes and the result are the
 * same bit for bit). This flag runs the split of every row as its own
 * kernels before the leaf instead. */
#define HPVM_LAUNCH_SEPARATE_SPLIT 256

typedef struct hpvm_ctx hpvm_ctx;
typedef struct hpvm_node hpvm_node;
typedef struct hpvm_edge hpvm_edge;
typedef struct hpvm_graph hpvm_graph;

/* ---- the argument record of the sgemm root ----------------------------
 * The first 88 bytes are the paper's packed %struct.RootIn (Section 6.1:
 * A, bytesA, lda, B, bytesB, ldb, C, bytesC, ldc, k, alpha, beta, block_x,
 * block_y, grid_x, grid_y; the host code mallocs 88 bytes and packs them).
 * Root input port p is field p of this record for p = 0..15; the trailer
 * adds M (port 16), N (17), transA (18), transB (19), which the example
 * leaves implicit, two launch options that are not graph inputs (tier,
 * flags), then aux (port 20), bytesAux (21), ldaux (22) for a leaf that
 * reads one more matrix (the H of TANH_GRAD_LEAF).
 * A launch passes an array of these records: port p of the root is field
 * p % 23 of record p / 23 (multi-stage graphs give each stage a record; at
 * most 16). The tier and flags of a stage come from the record holding its
 * C.
 *
 * Meaning: C <- alpha * op(A) * op(B) + beta * C with column-major storage
 * (element (r, c) of a matrix with leading dimension ld at r + c*ld);
 * op(A) = A (M x K, lda >= M) when transA == 0, else A^T (A stored K x M,
 * lda >= K); op(B) = B (K x N, ldb >= K) when transB == 0, else B^T (B
 * stored N x K, ldb >= N). The example's form is transA = 0, transB = 1.
 * C is M x N, ldc >= M. bytesX is the size of buffer X in bytes. When
 * beta == 0, C is not read. k = K. */
#pragma pack(push, 1)
typedef struct hpvm_sgemm_root_args {
  float* A;
  int64_t bytesA;
  int32_t lda;
  float* B;
  int64_t bytesB;
  int32_t ldb;
  float* C;
  int64_t bytesC;
  int32_t ldc;
  int32_t k;
  float alpha;
  float beta;
  int32_t block_x;
  int32_t block_y;
  int32_t grid_x;
  int32_t grid_y;
  /* trailer */
  int32_t M;
  int32_t N;
  int32_t transA;
  int32_t transB;
  int32_t tier;  /* HPVM_TIER_* */
  int32_t flags; /* HPVM_LAUNCH_* */
  float* aux;
  int64_t bytesAux;
  int32_t ldaux;
  int32_t reserved;
} hpvm_sgemm_root_args;
#pragma pack(pop)

#define HPVM_ROOTIN_PAPER_BYTES 88
#define HPVM_SGEMM_ROOT_ARGS_BYTES 136

/* What a launch ran (filled by hpvm_graph_info). */
typedef struct hpvm_launch_info {
  int32_t tier;
  int32_t kernels;       /* kernels launched for this graph */
  int32_t grid_x, grid_y, grid_z;  /* grid of the main (leaf) kernel */
  int32_t block_threads; /* threads per CTA of the main kernel */
  int32_t tile_m, tile_n, tile_k;  /* output tile per CTA, K slab */
  int32_t smem_bytes;    /* dynamic shared memory of the main kernel */
  int32_t literal;       /* 1: internal instance == CTA, leaf instance ==
                            thread (Section 3.4 mapping); 0: re-tiled */
  int64_t workspace_bytes;
  int64_t h2d_bytes, d2h_bytes; /* memory-tracker copies this launch made */
} hpvm_launch_info;

/* ---- runtime set-up (llvm.hpvm.init / llvm.hpvm.cleanup, Section 6.1) --
 * device >= 0: a context on that CUDA device (made current for the calling
 * thread). device < 0: a host-only context that can build and validate
 * graphs but not launch them (HPVM_ERR_NO_DEVICE from hpvm_launch). */
HPVM_API int hpvm_init(int device, hpvm_ctx** out);
/* Frees every node, edge, graph handle, tracked device copy and owned
 * workspace of the context, after synchronising its device. */
HPVM_API int hpvm_cleanup(hpvm_ctx* ctx);

/* ---- graph intrinsics (Table 1; Section 2.2 list) ----------------------
 * createNode / createNode{1,2,3}D: a child of `parent` (NULL for the root)
 * running node function `kind`, with `ndims` in 0..3 (0 = one instance) and
 * extents dims[0..ndims-1], each > 0 or HPVM_DIM_FROM_INPUT(p). Only an
 * internal node may be a parent. */
HPVM_API int hpvm_create_node(hpvm_ctx* ctx, hpvm_node* parent, int kind, int ndims,
                     const int64_t* dims, hpvm_node** out);
/* createEdge(Src, Dst, ReplTy, sp, dp, Stream): from output sp of src to
 * input dp of dst; both children of the same internal node; repl is
 * HPVM_ONE_TO_ONE or HPVM_ALL_TO_ALL; one-to-one needs identical grids.
 * stream != 0 makes it a streaming edge (items flow through it repeatedly,
 * Section 2.1); the lowering supports streaming edges between tile grids.
 * `out` may be NULL. */
HPVM_API int hpvm_create_edge(hpvm_node* src, hpvm_node* dst, int repl, int sp, int dp,
                     int stream, hpvm_edge** out);
/* bind.input(N, ip, ic, Stream): input ip of N's parent feeds input ic of N. */
HPVM_API int hpvm_bind_input(hpvm_node* child, int ip, int ic, int stream);
/* bind.output(N, oc, op, Stream): output oc of N becomes output op of its
 * parent. */
HPVM_API int hpvm_bind_output(hpvm_node* child, int oc, int op, int stream);

/* ---- query intrinsics, host side (Table 1) ----------------------------- */
HPVM_API int hpvm_get_parent_node(hpvm_node* node, hpvm_node** out); /* NULL for root */
HPVM_API int hpvm_get_num_dims(hpvm_node* node, int* out);
/* Static extent of dimension dim (or HPVM_DIM_FROM_INPUT(p)); dims beyond
 * the node's rank report 1. */
HPVM_API int hpvm_get_num_node_instances(hpvm_node* node, int dim, int64_t* out);

/* Check the graph under `root` against the rules of Sections 2.1-2.2:
 * root is a single-instance internal node; leaves have no children; edges
 * join siblings, ports are in range, one-to-one edges join equal grids, no
 * cycle of ordinary edges; every leaf input is fed exactly once. */
HPVM_API int hpvm_validate(hpvm_node* root);

/* ---- host integration (llvm.hpvm.launch / wait / push / pop) ----------
 * The lowered graph shapes: the root holds one or more 2-D internal nodes
 * (tile grids, one per stage, ordered by their edges: an all-to-all edge
 * from a stage's output 0 to the next stage's input carries the result
 * matrix); each holds one Allocation, one SgemmLeaf and at most one
 * elementwise leaf. When stage i + 1 reads stage i's result as its B
 * (op(B) = B, its K = stage i's M, the same BF16X3 or BF16 tier, merged,
 * no plane-cache flag on that B), stage i's epilogue also writes the BF16
 * planes stage i + 1 reads, and stage i + 1 converts no B (the planes equal
 * the converted ones bit for bit; HPVM_LAUNCH_NO_FUSION turns this off).
 * Launch the graph under `root` asynchronously on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream) with the argument records
 * `args` (hpvm_sgemm_root_args[], args_size >= 136). Errors found before any
 * work is enqueued (graph, shape, alignment) leave the stream untouched.
 * Launches of one context share its workspace (the tensor tiers' operand
 * planes and tail-split sums): a launch on a different stream than the
 * previous launch that used the workspace first waits for that launch (an
 * event), so the two do not overlap on the GPU. Inside CUDA stream capture
 * no such wait is added: captured launches of one context must be ordered
 * by the caller (one stream, or events of the capture).
 * stream_graph != 0 launches a streaming graph (Section 3.5): it is
 * validated against `args` and stays alive; nothing runs until items are
 * pushed. */
HPVM_API int hpvm_launch(hpvm_ctx* ctx, hpvm_node* root, const void* args,
                size_t args_size, int stream_graph, void* cuda_stream,
                hpvm_graph** out);
/* Wait until the launched graph finished, at most timeout_ms milliseconds
 * (< 0: no limit). HPVM_ERR_TIMEOUT leaves the handle valid; any other
 * return frees it. HPVM_ERR_DEVICE_FAULT: a kernel gave up a bounded wait
 * (the results are not valid). The status word that records such an expiry
 * belongs to the context, not to a graph: the first hpvm_wait or hpvm_pop
 * after the expiry reports it (and clears it), whichever graph of the
 * context it is called for, so with several graphs in flight treat the
 * error as "some launch of this context since the last check failed". */
HPVM_API int hpvm_wait(hpvm_graph* graph, int64_t timeout_ms);
/* Push one item into a streaming graph: `args` holds the item's records
 * (as for hpvm_launch). The item runs asynchronously on the next of the
 * graph's CUDA streams (4, round robin), so successive items overlap on
 * the GPU; every stream first waits for the work the caller's stream had
 * when the graph was launched. Items must not write the same buffers. The
 * graph's structure is validated at launch and again at a push only if a
 * node, edge or binding was added in the context since (an invalid graph
 * then gives HPVM_ERR_INVALID_GRAPH and nothing is enqueued). */
HPVM_API int hpvm_push(hpvm_graph* graph, const void* args, size_t args_size);
/* Pop the oldest pushed item: wait for it (at most timeout_ms, < 0: no
 * limit; HPVM_ERR_TIMEOUT leaves it queued), then copy its records into
 * out (up to out_size bytes) so the caller knows which buffers hold its
 * result. HPVM_ERR_INVALID_ARG when nothing was pushed. hpvm_wait on a
 * streaming graph waits for every item still queued and frees the graph. */
HPVM_API int hpvm_pop(hpvm_graph* graph, void* out, size_t out_size, int64_t timeout_ms);

/* Run up to `items` (>= 1) pushed items of a streaming graph as one
 * launch (no counterpart in the paper; its pipelined stages of Section 3.5
 * process items one at a time). With items > 1, hpvm_push queues an item
 * and enqueues nothing until `items` are queued; hpvm_pop of a queued item
 * and hpvm_wait launch whatever is queued. Queued items that share every
 * record field but the first stage's B, the last stage's C and their N
 * (the rows of the items: B is K x N with ldb = K, op(B) = B, C is M x N
 * with ldc = M), with beta = 0, no auxiliary matrix and device pointers,
 * run as one launch over the sum of their N: their B operands are used in
 * place when they lie side by side in memory (in push order), else copied
 * side by side into the slot's workspace; each stage runs once; the last
 * result is written in place when the items' C lie side by side, else
 * copied back to each item's C (the intermediate results of such a launch
 * go to the workspace, not to the items' buffers). Others run one launch
 * each. A push into a coalescing graph only queues the item (its records
 * are checked when its group is launched, and a bad record is reported by
 * the push, pop or wait that launches it). Each output is the same K sum as in a launch of its
 * item alone, bit for bit, except where the wider launch splits its last
 * round of tiles in K halves (many tiles, a short last round) and adds the
 * halves. 1 (the default) launches every item when it is pushed. */
HPVM_API int hpvm_stream_coalesce(hpvm_graph* graph, int items);
/* Copy the description of what `graph` launched into *out. */
HPVM_API int hpvm_graph_info(hpvm_graph* graph, hpvm_launch_info* out);

/* ---- memory tracker (Section 2.3) -------------------------------------
 * track_mem: host region [p, p+bytes) may be named in argument records; its
 * latest copy is the host's. A launch copies it to a device copy the
 * runtime owns when the copy there is stale and the leaf reads it (A, B;
 * C unless beta == 0), and marks C's latest copy as the device's.
 * request_mem: make the host copy of [p, p+bytes) current: waits for the
 * launch that last wrote the region (for the whole device when that launch
 * was captured into a CUDA graph), then copies device -> host if needed.
 * Launches on other streams, or of other contexts, keep running meanwhile.
 * untrack_mem: forget the region and free its device copy. */
HPVM_API int hpvm_track_mem(hpvm_ctx* ctx, void* p, int64_t bytes);
HPVM_API int hpvm_request_mem(hpvm_ctx* ctx, void* p, int64_t bytes);
HPVM_API int hpvm_untrack_mem(hpvm_ctx* ctx, void* p);

/* ---- workspace ----------------------------------------------------------
 * Device scratch the tensor-core tiers use: the operand planes of the
 * largest stage (for a BF16 or BF16x3 stage whose last round of pair tiles
 * splits in K halves, followed by their partial sums and arrival counters)
 * and, when stages forward planes to the next stage's B, two regions for
 * those. Bytes a launch of `root` with `args` needs: */
HPVM_API int hpvm_workspace_size(hpvm_ctx* ctx, hpvm_node* root, const void* args,
                        size_t args_size, size_t* out);
/* Use caller-owned device memory as workspace (NULL/0: the runtime
 * allocates and caches its own). Must stay valid while launches use it.
 * Launches on several streams are ordered as hpvm_launch describes; other
 * users of the same memory (another context, the caller's own kernels) are
 * not. */
HPVM_API int hpvm_set_workspace(hpvm_ctx* ctx, void* dev_ptr, size_t bytes);
/* The operand plane cache (HPVM_LAUNCH_CACHE_* / REUSE_*): its size in bytes,
 * and freeing it (after every launch that reads a cached plane has finished;
 * blocks the calling thread until then). */
HPVM_API int hpvm_plane_cache_bytes(hpvm_ctx* ctx, int64_t* bytes);
HPVM_API int hpvm_drop_planes(hpvm_ctx* ctx);

/* ---- planning -----------------------------------------------------------
 * Leaf instance grid and internal grid for an M x N result in `tier`:
 * the tile each kernel computes natively (block_x x block_y outputs per
 * internal instance) and the grid that covers M x N with it. */
HPVM_API int hpvm_plan_sgemm(int tier, int64_t M, int64_t N, int64_t K, int32_t* block_x,
                    int32_t* block_y, int32_t* grid_x, int32_t* grid_y);

/* ---- kernel timing ------------------------------------------------------
 * When enabled, every launch records CUDA events on its stream right before
 * and right after its main (leaf) kernel. hpvm_kernel_timing waits for the
 * recorded events, returns the summed main-kernel time in milliseconds and
 * the number of timed launches, and forgets them. */
HPVM_API int hpvm_set_kernel_timing(hpvm_ctx* ctx, int enable);
HPVM_API int hpvm_kernel_timing(hpvm_ctx* ctx, double* total_ms, int64_t* launches);

/* ---- operand preparation (the tensor-core tiers' pre-pass) ---------------
 * The first step of the BF16x3 / BF16 / FP8 leaves, callable on its own.
 * Y is a rows x K operand read from the column-major buffer X: element
 * (r, k) is X[r + k*ld] when kcontig == 0 (op(A) = A with rows = M, or
 * op(B) = B^T with rows = N), X[k + r*ld] when kcontig != 0 (op(A) = A^T, or
 * op(B) = B). Outputs are K-major, device pointers, 16-byte aligned;
 * asynchronous on cuda_stream.
 * hpvm_split_bf16: hi[r*Kp + k] = bf16_rn(Y(r,k)) and, when lo != NULL,
 *   lo[r*Kp + k] = bf16_rn(Y(r,k) - hi) (the difference is exact in FP32),
 *   with Kp = roundup(K, 8) and zeros for K <= k < Kp; hi, lo hold rows*Kp
 *   BF16 values.
 * hpvm_quant_fp8: for each 128 x 128 block (rb, kb) of Y, scales[rb*nkb + kb]
 *   = amax / 448 (1 for an all-zero block), nkb = ceil(K/128), both
 *   divisions IEEE FP32; q[r*Kq + k] = e4m3_rn_satfinite(Y(r,k) / scale) with
 *   Kq = roundup(K, 16) and zero codes for K <= k < Kq. */
HPVM_API int hpvm_split_bf16(const float* X, int64_t ld, int kcontig, int64_t rows, int64_t K,
                             void* hi, void* lo, void* cuda_stream);
/* hpvm_split3_bf16: the BF16X6 tier's pre-pass, three planes of rows*Kp
 *   BF16 values (Kp = roundup(K, 8), zeros for K <= k < Kp):
 *   hi[r*Kp + k] = bf16_rn(Y(r,k)), mid[...] = bf16_rn(Y(r,k) - hi) and
 *   lo[...] = bf16_rn(Y(r,k) - hi - mid), both differences exact in FP32. */
HPVM_API int hpvm_split3_bf16(const float* X, int64_t ld, int kcontig, int64_t rows, int64_t K,
                              void* hi, void* mid, void* lo, void* cuda_stream);
HPVM_API int hpvm_quant_fp8(const float* X, int64_t ld, int kcontig, int64_t rows, int64_t K,
                            void* q, float* scales, void* cuda_stream);

/* ---- allocation-free BF16x3 leaf ------------------------------------------
 * No counterpart in the paper. For callers that cannot allocate device
 * memory at call time -- code inside another framework's memory pool, code on
 * a latency-critical thread where cudaMalloc/cudaFree may synchronise the
 * device, code that must not run out of memory mid-job -- this computes
 * C <- alpha*op(A)*op(B) + beta*C exactly like the BF16X3 tier of
 * hpvm_launch (same kernels, same result), with the same column-major
 * argument meaning as hpvm_sgemm_root_args (transA/transB select op()), but
 * without a context, a graph or a workspace: the split BF16 planes live in a
 * fixed device array of HPVM_NOALLOC_SCRATCH_BYTES inside the library, which
 * every GPU that loads the library holds until the process exits.
 *   - A, B, C: device pointers owned by the caller; C is read (unless
 *     beta == 0) and written. dev_status: optional device-visible int the
 *     kernel ORs a nonzero bit into if one of its bounded waits expires (C is
 *     then not valid); NULL: not reported. cuda_stream: cudaStream_t, NULL =
 *     legacy default stream. The call is asynchronous on that stream.
 *   - It allocates nothing: no cudaMalloc, cudaFree or allocating library
 *     call. The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it, so make
 *     the first call on each device before any stream capture. Under CUDA's
 *     default lazy module loading that first lookup is also what loads the
 *     library's kernels onto the device and so creates the 64 MiB array
 *     there: make a first call (a small product will do) before a memory pool
 *     reserves the device's memory, or the array may not fit. After a
 *     cudaDeviceReset the device has a new context; the next call sees that
 *     and looks the address up again.
 *   - Every call uses the same array, and the array keeps the contents the
 *     last call left. The split planes a call reads, the same call writes
 *     first; the tail split's arrival counters (when its partial sums fit in
 *     the array) are zeroed by a cudaMemsetAsync that the call enqueues on
 *     its stream before the leaf kernel. Calls whose executions overlap on the
 *     GPU (concurrent streams, or several threads) race on the array and give
 *     wrong results: serialise them.
 *   - Errors: HPVM_ERR_SHAPE when the planes, 4*(M+N)*roundup(K,8) bytes with
 *     256-byte alignment per plane, exceed HPVM_NOALLOC_SCRATCH_BYTES (use
 *     hpvm_launch with a workspace then), or for a bad leading dimension;
 *     HPVM_ERR_INVALID_ARG for a NULL matrix; HPVM_ERR_CUDA if the launch
 *     fails. M == 0 or N == 0 is a no-op. */
#define HPVM_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
HPVM_API int hpvm_sgemm_bf16x3_noalloc(int64_t M, int64_t N, int64_t K, float alpha,
                                       const float* A, int64_t lda, const float* B, int64_t ldb,
                                       float beta, float* C, int64_t ldc, int transA, int transB,
                                       int* dev_status, void* cuda_stream);

/* ---- batches of independent DFG instances -----------------------------
 * No paper counterpart: many instances of one single-stage sgemm graph
 * (records[i] = instance i's argument records, record_bytes apart), run by
 * one split pre-pass launch and one persistent launch of the grouped leaf
 * over every output tile of every instance, longest tiles first.
 * Instances take the BF16X3 or BF16 tier (the same for all) and device
 * pointers. The hierarchy of every instance (Section 3.4 leaves tile sizes
 * to an autotuner) comes from a policy: its tile height, 128 rows on one
 * persistent CTA (policies 0-3) or 256 rows on a persistent CTA pair of a
 * cluster (4-7; 8-11 the same, BF16X3 only, with the operand planes made
 * inside the leaf: the pre-pass splits only what the leaf's first round of
 * tiles reads, and idle warps of the leaf convert the rest, in the order
 * the tiles first read it), and each instance's tile width (its leaf grid,
 * block_y = 64, 128 or 256 columns per internal instance) by the rule
 * policy & 3:
 *   0: 256 for all; 1: 128 for all; 2, 3: per instance, the width that
 *   minimises tiles x (width x padded K + overhead), overhead light (2) or
 *   heavy (3). -1: the policy hpvm_batch_autotune found for a batch of the
 *   same shapes in this context, else 2.
 * prepare allocates the batch's operand planes and tables on the device
 * (runtime-owned, freed by hpvm_batch_free or hpvm_cleanup) and sets kernel
 * attributes; run only enqueues the two kernels (8-11: a reset of the
 * conversion's flags too), so it can be captured in
 * a CUDA graph. A batch reads the pointers of its records at every run. */
typedef struct hpvm_batch hpvm_batch;
typedef struct hpvm_batch_stats {
  int32_t count, tier, policy;
  int32_t tiles;        /* output tiles of the leaf launch */
  int32_t split_tiles;  /* 64 x 64 tiles of the pre-pass launch (8-11: the first round's) */
  int32_t grid;         /* persistent CTAs */
  int32_t tile_width_count[3]; /* instances with 64, 128, 256 columns */
  int32_t tile_m;       /* rows of an output tile: 128 or 256 (CTA pairs) */
  int64_t workspace_bytes;
} hpvm_batch_stats;
HPVM_API int hpvm_batch_prepare(hpvm_ctx* ctx, hpvm_node* root, const void* records, size_t record_bytes,
                                int count, int policy, hpvm_batch** out);
HPVM_API int hpvm_batch_run(hpvm_batch* batch, void* cuda_stream);
/* Time each policy, 0..11 (0..7 for BF16) (reps runs after one warm-up, CUDA events on
 * cuda_stream), keep the fastest for this batch and for later batches of
 * the same shapes in the context. Results of the timed runs are valid. */
HPVM_API int hpvm_batch_autotune(hpvm_batch* batch, void* cuda_stream, int reps, int* best_policy,
                                 double* best_ms);
HPVM_API int hpvm_batch_info(hpvm_batch* batch, hpvm_batch_stats* out);
HPVM_API int hpvm_batch_free(hpvm_batch* batch);
/* Host-only: the tile widths a policy (0..11) picks for instances of the
 * given shapes, and the leaf's schedule in launch order, 4 ints per slot
 * (instance, m0, n0, unit): tiles (128 rows, or 256 for policies 4-11) go
 * longest first to the persistent unit (a CTA, or a CTA pair) with the
 * least work so far, unit u runs slots u, u + G, u + 2G, ... (G = the
 * units, at most the current device's SMs, or half of them for pairs), and
 * a unit with fewer tiles than the busiest has empty slots (instance -1).
 * tiles may be NULL to query num_tiles (the slot count). */
HPVM_API int hpvm_batch_plan(int count, const int64_t* M, const int64_t* N, const int64_t* K, int policy,
                             int32_t* bn, int32_t* tiles, int64_t tile_cap, int64_t* num_tiles);

/* ---- failure detection self-test ---------------------------------------
 * No paper counterpart. Runs one kernel whose single mbarrier wait nothing
 * ever satisfies, through the same bounded wait the leaf kernels use, with
 * a limit of limit_ms (1..10000). The wait gives up, the kernel records it
 * in the context's status word and returns; this call waits for it and
 * returns what a graph's hpvm_wait would: HPVM_ERR_DEVICE_FAULT. No copy,
 * MMA or tensor memory is involved and the context stays usable. */
HPVM_API int hpvm_selftest_wait_timeout(hpvm_ctx* ctx, int64_t limit_ms, void* cuda_stream);

/* Limit of each bounded wait inside the tensor-core leaves of this
 * context's later launches, in microseconds (0: the default of 2 s;
 * 1..10^7). No paper counterpart. A wait that runs past it gives up: the
 * kernel records it in the status word, stops every role, waits (bounded
 * by the default) for the copies and MMAs it started, frees its tensor
 * memory and returns, and hpvm_wait reports HPVM_ERR_DEVICE_FAULT. A short
 * limit makes the waits of a normal launch run out, which is how the
 * failure path is tested; the context stays usable. */
HPVM_API int hpvm_set_wait_limit(hpvm_ctx* ctx, int64_t limit_us);

/* Thread-local message of the last failed call ("" if none). */
HPVM_API const char* hpvm_last_error(void);
/* ABI version (major * 100 + minor). */
HPVM_API int hpvm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HPVM_GB300_HPVM_H */
