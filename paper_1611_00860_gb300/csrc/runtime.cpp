// Host runtime of the C-ABI (include/hpvm.h).
//
//  * Graph builder (the paper's Graph Builder pass, Section 3.2, fed by the
//    intrinsic calls of Table 1 instead of IR) and validator (the rules of
//    Sections 2.1-2.2).
//  * Lowering (Sections 3.3-3.4 and the generated host code of Section 6.3):
//    every input of a leaf is resolved by following edges and bindings up to
//    a field of the root's argument records; the Allocation size is computed
//    on the host before the launch; each tile-grid stage becomes one leaf
//    kernel launch, with a dependent elementwise leaf merged into the
//    kernel's epilogue (MergeDependentNodes, Section 4.1) or run after it.
//  * Launch and bounded wait; streaming graphs (Section 3.5) whose items are
//    pushed and popped, pipelined over a ring of CUDA streams.
//  * The memory tracker of Section 2.3.
//  * The operand plane cache (no counterpart in the paper): the BF16 / E4M3
//    planes of an operand kept across launches (CACHE_* / REUSE_* flags),
//    filled by a conversion or, for a stage's result, by its epilogue
//    (CACHE_C; with PLANES_ONLY the result is kept only as planes).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hpvm.h"
#include "internal.h"

// ---------------------------------------------------------------------------
// errors
namespace {
thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  return fail(HPVM_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}
int ok() {
  g_last_error.clear();
  return HPVM_OK;
}

constexpr int kMaxPorts = 64;  // ports of an internal node below the root

// The root's argument records: port p of the root is field p % kRecPorts of
// record p / kRecPorts (one record per stage of a multi-stage graph).
enum FieldType { F_PTR, F_I64, F_I32, F_F32 };
constexpr int kRecPorts = 23;
constexpr int kMaxRecords = 16;
constexpr int kRootPorts = kRecPorts * kMaxRecords;
constexpr size_t kRecBytes = HPVM_SGEMM_ROOT_ARGS_BYTES;
constexpr FieldType kRecType[kRecPorts] = {
    F_PTR, F_I64, F_I32,          // A, bytesA, lda
    F_PTR, F_I64, F_I32,          // B, bytesB, ldb
    F_PTR, F_I64, F_I32,          // C, bytesC, ldc
    F_I32, F_F32, F_F32,          // k, alpha, beta
    F_I32, F_I32, F_I32, F_I32,   // block_x, block_y, grid_x, grid_y
    F_I32, F_I32, F_I32, F_I32,   // M, N, transA, transB
    F_PTR, F_I64, F_I32,          // aux, bytesAux, ldaux
};
constexpr size_t kRecOffset[kRecPorts] = {0,  8,  16, 20, 28, 36, 40, 48, 56, 60, 64, 68,
                                          72, 76, 80, 84, 88, 92, 96, 100, 112, 120, 128};
constexpr size_t kTierOffset = 104, kFlagsOffset = 108;
const char* kRecName[kRecPorts] = {"A",       "bytesA",  "lda",    "B",      "bytesB", "ldb",
                                   "C",       "bytesC",  "ldc",    "k",      "alpha",  "beta",
                                   "block_x", "block_y", "grid_x", "grid_y", "M",      "N",
                                   "transA",  "transB",  "aux",    "bytesAux", "ldaux"};

// Input ports of the leaf node functions and their types.
constexpr int kLeafPorts = 20;
constexpr FieldType kLeafType[kLeafPorts] = {
    F_PTR, F_I64, F_I32, F_PTR, F_I64, F_I32, F_PTR, F_I64, F_I32,  // A..ldc
    F_I32, F_F32, F_F32,                                            // k, alpha, beta
    F_PTR, F_I64, F_PTR, F_I64,  // shB, bytesShB, shA, bytesShA (Allocation)
    F_I32, F_I32, F_I32, F_I32,  // M, N, transA, transB
};
constexpr int kTanhPorts = 5;      // X, bytesX, ldx, M, N
constexpr int kTanhGradPorts = 8;  // G, bytesG, ldg, M, N, H, bytesH, ldh
constexpr FieldType kEwType[kTanhGradPorts] = {F_PTR, F_I64, F_I32, F_I32, F_I32, F_PTR, F_I64, F_I32};
constexpr int kAllocInPorts = 2, kAllocOutPorts = 4;
constexpr FieldType kAllocOutType[kAllocOutPorts] = {F_PTR, F_I64, F_PTR, F_I64};
constexpr int kStreamSlots = 4;  // CUDA streams of a streaming graph

const char* kind_name(int k) {
  switch (k) {
    case HPVM_NODE_INTERNAL: return "internal";
    case HPVM_NODE_ALLOCATION: return "Allocation";
    case HPVM_NODE_SGEMM_LEAF: return "SgemmLeaf";
    case HPVM_NODE_TANH_LEAF: return "TanhLeaf";
    case HPVM_NODE_TANH_GRAD_LEAF: return "TanhGradLeaf";
  }
  return "?";
}
}  // namespace

int hpvm::set_last_error(int code, const char* msg) {
  if (code == HPVM_OK) return ok();
  return fail(code, "%s", msg);
}

// ---------------------------------------------------------------------------
// handles
struct hpvm_edge {
  hpvm_node* src;
  hpvm_node* dst;
  int repl, sp, dp, stream;
};

// in_binds: input `outer` of the parent feeds input `inner` of child.
// out_binds: output `inner` of child becomes output `outer` of the parent.
struct Bind {
  hpvm_node* child;
  int outer, inner, stream;
};

struct hpvm_node {
  hpvm_ctx* ctx = nullptr;
  hpvm_node* parent = nullptr;
  int kind = 0;
  int ndims = 0;
  int64_t dims[3] = {1, 1, 1};
  int id = 0;
  std::vector<hpvm_node*> children;
  std::vector<hpvm_edge*> edges;   // among children
  std::vector<Bind> in_binds;
  std::vector<Bind> out_binds;
};

struct TrackEntry {
  char* host = nullptr;
  int64_t bytes = 0;
  void* dev = nullptr;
  bool host_valid = true, dev_valid = false;
  // recorded after the last launch that wrote the device copy (unset when
  // that launch was captured into a CUDA graph)
  cudaEvent_t written = nullptr;
  bool written_set = false;
};

// one pushed item of a streaming graph (launched: enqueued on a stream;
// not yet when it waits to run together with later items)
struct StreamItem {
  std::vector<uint8_t> record;
  cudaEvent_t done = nullptr;
  bool launched = false;
};

struct hpvm_graph {
  hpvm_ctx* ctx = nullptr;
  cudaEvent_t done = nullptr;
  cudaStream_t stream = nullptr;
  hpvm_launch_info info{};
  // streaming graphs
  bool streaming = false;
  hpvm_node* root = nullptr;
  std::vector<cudaStream_t> slots;
  std::vector<void*> slot_ws;
  std::vector<size_t> slot_ws_bytes;
  std::deque<StreamItem> items;
  std::vector<cudaEvent_t> spare_events;  // events of popped items, reused
  uint64_t pushed = 0;    // items pushed (slot of the next per-item launch)
  uint64_t launches = 0;  // launches made for items (one per item, or per coalesced group)
  int coalesce = 1;       // queued items run as one launch once this many wait
  uint64_t validated = ~uint64_t(0);  // the context's structure version validated at launch
};

struct hpvm_batch {
  hpvm_ctx* ctx = nullptr;
  hpvm::TcBatch tb;
  uint64_t signature = 0;
};

// One operand's planes in the context's plane cache (HPVM_LAUNCH_CACHE_* /
// REUSE_*): the key, the device buffer, whether it holds the operand, the
// event recorded after its conversion, and per stream the event recorded
// after the last launch there that read it (a refill waits for those).
struct PlaneEntry {
  const void* src = nullptr;
  int64_t ld = 0, rows = 0, K = 0;
  int layout = 0, tier = 0;
  void* buf = nullptr;
  size_t bytes = 0;
  bool valid = false;
  cudaStream_t filled_on = nullptr;
  cudaEvent_t converted = nullptr;
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> uses;
};
constexpr size_t kPlaneCacheLimit = size_t(4) << 30;

struct hpvm_ctx {
  int device = -1;
  int next_id = 0;
  std::vector<std::unique_ptr<hpvm_node>> nodes;
  std::vector<std::unique_ptr<hpvm_edge>> edges;
  std::set<hpvm_graph*> graphs;
  std::vector<TrackEntry> tracked;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  // the last launch that used the workspace: its stream and an event
  // recorded after it (a launch on another stream waits for it)
  cudaStream_t ws_stream = nullptr;
  cudaEvent_t ws_event = nullptr;
  hpvm::DeviceStatus status;
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> timed;  // main-kernel events
  std::set<hpvm_batch*> batches;
  std::vector<std::pair<uint64_t, int>> tuned;  // batch shape signature -> best policy
  std::vector<std::unique_ptr<PlaneEntry>> planes;  // the operand plane cache
  size_t plane_bytes = 0;
  // bumped by every call that changes a graph (nodes, edges, bindings): a
  // streaming graph validated at launch is not validated again per push
  // unless this moved
  uint64_t structure = 0;
  cudaStream_t copy_stream = nullptr;  // request_mem's device -> host copies
  // streams and slot workspaces of finished streaming graphs, kept for the
  // next streaming graph (a streaming graph per batch of items would
  // otherwise create streams and allocate workspace every time)
  std::vector<cudaStream_t> spare_streams;
  std::vector<std::pair<void*, size_t>> spare_ws;
  std::vector<cudaEvent_t> spare_events;
};

// ---------------------------------------------------------------------------
// helpers
namespace {

bool is_leaf(const hpvm_node* n) { return n->kind != HPVM_NODE_INTERNAL; }
bool is_elementwise(const hpvm_node* n) {
  return n->kind == HPVM_NODE_TANH_LEAF || n->kind == HPVM_NODE_TANH_GRAD_LEAF;
}

int in_arity(const hpvm_node* n) {
  switch (n->kind) {
    case HPVM_NODE_SGEMM_LEAF: return kLeafPorts;
    case HPVM_NODE_ALLOCATION: return kAllocInPorts;
    case HPVM_NODE_TANH_LEAF: return kTanhPorts;
    case HPVM_NODE_TANH_GRAD_LEAF: return kTanhGradPorts;
    default: return n->parent == nullptr ? kRootPorts : kMaxPorts;
  }
}
int out_arity(const hpvm_node* n) {
  switch (n->kind) {
    case HPVM_NODE_SGEMM_LEAF: return 2;  // the result matrix C and its bytes
    case HPVM_NODE_ALLOCATION: return kAllocOutPorts;
    case HPVM_NODE_TANH_LEAF:
    case HPVM_NODE_TANH_GRAD_LEAF: return 2;  // the matrix it updated, bytes
    default: return kMaxPorts;
  }
}

std::string node_label(const hpvm_node* n) {
  char b[64];
  snprintf(b, sizeof b, "%s#%d", kind_name(n->kind), n->id);
  return b;
}

// How many times each input port of `child` is fed (edges + bindings).
std::vector<int> feed_counts(const hpvm_node* child) {
  std::vector<int> cnt(in_arity(child), 0);
  const hpvm_node* par = child->parent;
  if (!par) return cnt;
  for (auto* e : par->edges)
    if (e->dst == child && e->dp < (int)cnt.size()) cnt[e->dp]++;
  for (auto& b : par->in_binds)
    if (b.child == child && b.inner < (int)cnt.size()) cnt[b.inner]++;
  return cnt;
}

// ports of `n` that something under it reads (bindings to its children and
// replication extents of its children)
std::vector<bool> used_inputs(const hpvm_node* n) {
  std::vector<bool> used(in_arity(n), false);
  for (auto& b : n->in_binds)
    if (b.outer >= 0 && b.outer < (int)used.size()) used[b.outer] = true;
  for (auto* c : n->children)
    for (int d = 0; d < c->ndims; ++d)
      if (c->dims[d] < 0) {
        int64_t p = -1 - c->dims[d];
        if (p < (int64_t)used.size()) used[p] = true;
      }
  return used;
}

int index_of(const hpvm_node* parent, const hpvm_node* c) {
  for (size_t i = 0; i < parent->children.size(); ++i)
    if (parent->children[i] == c) return (int)i;
  return -1;
}

// Children of n in an order compatible with its edges; fails on a cycle.
int topo_children(const hpvm_node* n, std::vector<hpvm_node*>* order) {
  const size_t m = n->children.size();
  std::vector<int> indeg(m, 0);
  for (auto* e : n->edges) {
    int v = index_of(n, e->dst);
    if (v >= 0) indeg[v]++;
  }
  std::deque<int> ready;
  for (size_t i = 0; i < m; ++i)
    if (indeg[i] == 0) ready.push_back((int)i);
  order->clear();
  while (!ready.empty()) {
    int u = ready.front();
    ready.pop_front();
    order->push_back(n->children[u]);
    for (auto* e : n->edges)
      if (e->src == n->children[u]) {
        int v = index_of(n, e->dst);
        if (v >= 0 && --indeg[v] == 0) ready.push_back(v);
      }
  }
  if (order->size() != m) return fail(HPVM_ERR_INVALID_GRAPH, "cycle of edges under %s", node_label(n).c_str());
  return HPVM_OK;
}

int validate_node(const hpvm_node* n) {
  if (is_leaf(n)) {
    if (!n->children.empty())
      return fail(HPVM_ERR_INVALID_GRAPH, "%s: a leaf node has children", node_label(n).c_str());
    return HPVM_OK;
  }
  for (auto* e : n->edges) {
    if (e->src->parent != n || e->dst->parent != n)
      return fail(HPVM_ERR_INVALID_GRAPH, "edge endpoints are not children of %s", node_label(n).c_str());
    if (e->repl == HPVM_ONE_TO_ONE) {
      bool same = e->src->ndims == e->dst->ndims;
      for (int d = 0; same && d < e->src->ndims; ++d) same = e->src->dims[d] == e->dst->dims[d];
      if (!same)
        return fail(HPVM_ERR_INVALID_GRAPH,
                    "one-to-one edge %s -> %s joins grids of different rank or extent",
                    node_label(e->src).c_str(), node_label(e->dst).c_str());
    }
  }
  std::vector<hpvm_node*> order;
  int rc = topo_children(n, &order);
  if (rc != HPVM_OK) return rc;
  for (auto* c : n->children) {
    auto cnt = feed_counts(c);
    if (is_leaf(c)) {
      for (int p = 0; p < (int)cnt.size(); ++p) {
        if (cnt[p] == 0)
          return fail(HPVM_ERR_INVALID_GRAPH, "input %d of %s is not fed by an edge or a binding", p,
                      node_label(c).c_str());
        if (cnt[p] > 1)
          return fail(HPVM_ERR_INVALID_GRAPH, "input %d of %s is fed %d times", p, node_label(c).c_str(),
                      cnt[p]);
      }
    } else {
      auto used = used_inputs(c);
      for (int p = 0; p < (int)cnt.size(); ++p) {
        if (p < (int)used.size() && used[p] && cnt[p] == 0)
          return fail(HPVM_ERR_INVALID_GRAPH, "input %d of %s is read but never fed", p,
                      node_label(c).c_str());
        if (cnt[p] > 1)
          return fail(HPVM_ERR_INVALID_GRAPH, "input %d of %s is fed %d times", p, node_label(c).c_str(),
                      cnt[p]);
      }
    }
    rc = validate_node(c);
    if (rc != HPVM_OK) return rc;
  }
  return HPVM_OK;
}

// ---- value resolution -------------------------------------------------------
// Where a value comes from: a field of a root record, or an output of an
// Allocation node. Outputs of compute leaves and stages pass their inputs
// through (the matrix a leaf wrote), so every value resolves to one of the two.
struct Source {
  int rec = -1, field = -1;
  hpvm_node* alloc = nullptr;
  int alloc_out = -1;
};

bool input_source(const hpvm_node* n, int port, Source* out, int depth = 0);

bool value_of_input(const hpvm_node* n, int port, Source* out, int depth) {
  if (n->parent == nullptr) {
    if (port < 0 || port >= kRootPorts) return false;
    out->rec = port / kRecPorts;
    out->field = port % kRecPorts;
    return true;
  }
  return input_source(n, port, out, depth + 1);
}

bool output_source(const hpvm_node* n, int port, Source* out, int depth) {
  if (depth > 64) return false;
  switch (n->kind) {
    case HPVM_NODE_SGEMM_LEAF:
      return (port == 0 || port == 1) && input_source(n, 6 + port, out, depth + 1);
    case HPVM_NODE_TANH_LEAF:
    case HPVM_NODE_TANH_GRAD_LEAF:
      return (port == 0 || port == 1) && input_source(n, port, out, depth + 1);
    case HPVM_NODE_ALLOCATION:
      out->alloc = const_cast<hpvm_node*>(n);
      out->alloc_out = port;
      return true;
    default:
      for (auto& b : n->out_binds)
        if (b.outer == port) return output_source(b.child, b.inner, out, depth + 1);
      return false;
  }
}

bool input_source(const hpvm_node* n, int port, Source* out, int depth) {
  if (depth > 64) return false;
  const hpvm_node* par = n->parent;
  if (!par) return value_of_input(n, port, out, depth);
  for (auto* e : par->edges)
    if (e->dst == n && e->dp == port) return output_source(e->src, e->sp, out, depth + 1);
  for (auto& b : par->in_binds)
    if (b.child == n && b.inner == port) return value_of_input(par, b.outer, out, depth + 1);
  return false;
}

struct Records {
  const uint8_t* base;
  int count;
  template <class T>
  T get(int rec, int field) const {
    T v;
    memcpy(&v, base + rec * kRecBytes + kRecOffset[field], sizeof(T));
    return v;
  }
};

// Read a resolved root field of the expected type.
int read_field(const Records& R, const Source& s, FieldType want, const char* who, int port, int64_t* i,
               double* f, void** p) {
  if (s.rec < 0 || s.field < 0)
    return fail(HPVM_ERR_UNSUPPORTED, "%s input %d must come from the root records", who, port);
  if (s.rec >= R.count)
    return fail(HPVM_ERR_INVALID_ARG, "%s input %d reads record %d, only %d records were passed", who, port, s.rec,
                R.count);
  if (kRecType[s.field] != want)
    return fail(HPVM_ERR_INVALID_GRAPH, "%s input %d is bound to root field %s of another type", who, port,
                kRecName[s.field]);
  switch (want) {
    case F_PTR: *p = R.get<void*>(s.rec, s.field); break;
    case F_I64: *i = R.get<int64_t>(s.rec, s.field); break;
    case F_I32: *i = R.get<int32_t>(s.rec, s.field); break;
    case F_F32: *f = R.get<float>(s.rec, s.field); break;
  }
  return HPVM_OK;
}

bool extent_of(const hpvm_node* n, int d, const Records& R, int64_t* out) {
  if (d >= n->ndims) {
    *out = 1;
    return true;
  }
  if (n->dims[d] > 0) {
    *out = n->dims[d];
    return true;
  }
  Source s;
  if (!value_of_input(n->parent, (int)(-1 - n->dims[d]), &s, 0) || s.rec < 0 || s.rec >= R.count) return false;
  if (kRecType[s.field] != F_I32) return false;
  *out = R.get<int32_t>(s.rec, s.field);
  return true;
}

// One lowered tile-grid stage: a sgemm leaf and its merged elementwise leaf.
struct Stage {
  hpvm::SgemmDesc d;
  int64_t bytesA = 0, bytesB = 0, bytesC = 0;
  int64_t block_x = 0, block_y = 0, grid_x = 0, grid_y = 0;
  int64_t alloc_bx = 0, alloc_by = 0;
  bool has_a_tile = false;
  hpvm::Epilogue epi;
  int64_t bytesAux = 0;
  int rec = 0;  // the record (holding C) whose tier and flags apply
};

int64_t need_bytes(int64_t rows, int64_t cols, int64_t ld) {
  return (rows == 0 || cols == 0) ? 0 : 4 * (ld * (cols - 1) + rows);
}

int lower_stage(hpvm_node* stage, const Records& R, Stage* S) {
  hpvm_node* alloc = nullptr;
  hpvm_node* leaf = nullptr;
  hpvm_node* ew = nullptr;
  for (auto* c : stage->children) {
    if (c->kind == HPVM_NODE_ALLOCATION && !alloc) alloc = c;
    else if (c->kind == HPVM_NODE_SGEMM_LEAF && !leaf) leaf = c;
    else if (is_elementwise(c) && !ew) ew = c;
    else
      return fail(HPVM_ERR_UNSUPPORTED,
                  "a tile node must hold one Allocation, one SgemmLeaf and at most one elementwise leaf");
  }
  if (!alloc || !leaf) return fail(HPVM_ERR_UNSUPPORTED, "a tile node must hold one Allocation and one SgemmLeaf");
  if (alloc->ndims != 0) return fail(HPVM_ERR_UNSUPPORTED, "the Allocation node must have one instance");
  if (leaf->ndims != 2) return fail(HPVM_ERR_UNSUPPORTED, "the SgemmLeaf must be a 2-D grid");
  for (auto* e : stage->edges) {
    if (e->stream) return fail(HPVM_ERR_UNSUPPORTED, "streaming edges inside a tile node are not lowered");
    const bool alloc_edge = e->src == alloc && e->dst == leaf && e->repl == HPVM_ALL_TO_ALL;
    // MergeDependentNodes precondition: the elementwise leaf is joined to the
    // sgemm leaf only by one-to-one edges, result -> operand
    const bool merge_edge = ew && e->src == leaf && e->dst == ew && e->repl == HPVM_ONE_TO_ONE && e->sp == e->dp &&
                            (e->sp == 0 || e->sp == 1);
    if (!alloc_edge && !merge_edge)
      return fail(HPVM_ERR_UNSUPPORTED,
                  "only all-to-all Allocation -> SgemmLeaf and one-to-one SgemmLeaf -> elementwise edges are lowered");
  }
  for (auto& b : stage->in_binds)
    if (b.stream) return fail(HPVM_ERR_UNSUPPORTED, "streaming bindings inside a tile node are not lowered");

  int64_t vi[kLeafPorts] = {0};
  double vf[kLeafPorts] = {0};
  void* vp[kLeafPorts] = {nullptr};
  int rec = -1;
  int rc;
  for (int p = 0; p < kLeafPorts; ++p) {
    Source s;
    if (!input_source(leaf, p, &s))
      return fail(HPVM_ERR_INVALID_GRAPH,
                  "SgemmLeaf input %d does not resolve to a root field or an Allocation output", p);
    if (p >= 12 && p <= 15) {
      if (!s.alloc || s.alloc != alloc)
        return fail(HPVM_ERR_UNSUPPORTED, "SgemmLeaf input %d (tile memory) must come from the Allocation node", p);
      if (kAllocOutType[s.alloc_out] != kLeafType[p])
        return fail(HPVM_ERR_INVALID_GRAPH, "Allocation output %d has the wrong type for SgemmLeaf input %d",
                    s.alloc_out, p);
      if ((p == 12 && s.alloc_out != 0) || (p == 13 && s.alloc_out != 1))
        return fail(HPVM_ERR_UNSUPPORTED, "SgemmLeaf inputs 12, 13 must be Allocation outputs 0, 1");
      if (p == 14 || p == 15) S->has_a_tile = true;
      continue;
    }
    if ((rc = read_field(R, s, kLeafType[p], "SgemmLeaf", p, &vi[p], &vf[p], &vp[p])) != HPVM_OK) return rc;
    if (p == 6) rec = s.rec;
  }
  S->rec = rec < 0 ? 0 : rec;
  for (int p = 0; p < kAllocInPorts; ++p) {
    Source s;
    if (!input_source(alloc, p, &s)) return fail(HPVM_ERR_INVALID_GRAPH, "Allocation input %d is not fed", p);
    int64_t v = 0;
    double f;
    void* q;
    if ((rc = read_field(R, s, F_I32, "Allocation", p, &v, &f, &q)) != HPVM_OK) return rc;
    (p == 0 ? S->alloc_bx : S->alloc_by) = v;
  }
  if (!extent_of(leaf, 0, R, &S->block_x) || !extent_of(leaf, 1, R, &S->block_y) ||
      !extent_of(stage, 0, R, &S->grid_x) || !extent_of(stage, 1, R, &S->grid_y))
    return fail(HPVM_ERR_INVALID_GRAPH, "a replication extent does not resolve to an i32 root field");

  auto& d = S->d;
  d.A = static_cast<const float*>(vp[0]);
  S->bytesA = vi[1];
  d.lda = vi[2];
  d.B = static_cast<const float*>(vp[3]);
  S->bytesB = vi[4];
  d.ldb = vi[5];
  d.C = static_cast<float*>(vp[6]);
  S->bytesC = vi[7];
  d.ldc = vi[8];
  d.K = vi[9];
  d.alpha = (float)vf[10];
  d.beta = (float)vf[11];
  d.M = vi[16];
  d.N = vi[17];
  d.transA = vi[18] != 0;
  d.transB = vi[19] != 0;

  if (ew) {
    // the merged leaf must update exactly the sgemm result
    int64_t ei[kTanhGradPorts] = {0};
    double ef;
    void* ep[kTanhGradPorts] = {nullptr};
    const int np = ew->kind == HPVM_NODE_TANH_LEAF ? kTanhPorts : kTanhGradPorts;
    for (int p = 0; p < np; ++p) {
      Source s;
      if (!input_source(ew, p, &s))
        return fail(HPVM_ERR_INVALID_GRAPH, "%s input %d does not resolve", kind_name(ew->kind), p);
      if ((rc = read_field(R, s, kEwType[p], kind_name(ew->kind), p, &ei[p], &ef, &ep[p])) != HPVM_OK) return rc;
    }
    if (ep[0] != vp[6] || ei[2] != d.ldc || ei[3] != d.M || ei[4] != d.N)
      return fail(HPVM_ERR_UNSUPPORTED, "the elementwise leaf must update the sgemm leaf's own M x N result");
    S->epi.kind = ew->kind == HPVM_NODE_TANH_LEAF ? 1 : 2;
    if (S->epi.kind == 2) {
      S->epi.aux = static_cast<const float*>(ep[5]);
      S->bytesAux = ei[6];
      S->epi.ldaux = ei[7];
      if (S->epi.ldaux < std::max<int64_t>(1, d.M))
        return fail(HPVM_ERR_SHAPE, "ldh (%lld) < M", (long long)S->epi.ldaux);
      if (d.M > 0 && d.N > 0 && (!S->epi.aux || S->bytesAux < need_bytes(d.M, d.N, S->epi.ldaux)))
        return fail(HPVM_ERR_SHAPE, "H is NULL or smaller than M x N with ldh");
    }
  }

  // shapes
  if (d.M < 0 || d.N < 0 || d.K < 0) return fail(HPVM_ERR_SHAPE, "negative M, N or K");
  if (S->block_x <= 0 || S->block_y <= 0 || S->grid_x <= 0 || S->grid_y <= 0)
    return fail(HPVM_ERR_SHAPE, "replication extents must be positive");
  if (S->grid_x * S->block_x < d.M || S->grid_y * S->block_y < d.N)
    return fail(HPVM_ERR_SHAPE, "grid x block (%lld x %lld) does not cover M x N (%lld x %lld)",
                (long long)(S->grid_x * S->block_x), (long long)(S->grid_y * S->block_y), (long long)d.M,
                (long long)d.N);
  const int64_t ar = d.transA ? d.K : d.M, ac = d.transA ? d.M : d.K;
  const int64_t br = d.transB ? d.N : d.K, bc = d.transB ? d.K : d.N;
  if (d.lda < std::max<int64_t>(1, ar))
    return fail(HPVM_ERR_SHAPE, "lda (%lld) < rows of A (%lld)", (long long)d.lda, (long long)ar);
  if (d.ldb < std::max<int64_t>(1, br))
    return fail(HPVM_ERR_SHAPE, "ldb (%lld) < rows of B (%lld)", (long long)d.ldb, (long long)br);
  if (d.ldc < std::max<int64_t>(1, d.M))
    return fail(HPVM_ERR_SHAPE, "ldc (%lld) < M (%lld)", (long long)d.ldc, (long long)d.M);
  const bool work = d.M > 0 && d.N > 0;
  if (work && d.K > 0) {
    if (!d.A || !d.B) return fail(HPVM_ERR_INVALID_ARG, "A or B is NULL");
    if (S->bytesA < need_bytes(ar, ac, d.lda))
      return fail(HPVM_ERR_SHAPE, "bytesA (%lld) < %lld needed", (long long)S->bytesA, (long long)need_bytes(ar, ac, d.lda));
    if (S->bytesB < need_bytes(br, bc, d.ldb))
      return fail(HPVM_ERR_SHAPE, "bytesB (%lld) < %lld needed", (long long)S->bytesB, (long long)need_bytes(br, bc, d.ldb));
  }
  if (work) {
    if (!d.C) return fail(HPVM_ERR_INVALID_ARG, "C is NULL");
    if (S->bytesC < need_bytes(d.M, d.N, d.ldc))
      return fail(HPVM_ERR_SHAPE, "bytesC (%lld) < %lld needed", (long long)S->bytesC, (long long)need_bytes(d.M, d.N, d.ldc));
  }
  return HPVM_OK;
}

struct Plan {
  std::vector<Stage> stages;
  Records R{nullptr, 0};
};

int lower_graph(hpvm_node* root, const void* args, size_t args_size, Plan* P, bool validated = false) {
  if (!root || root->parent != nullptr)
    return fail(HPVM_ERR_INVALID_ARG, "launch needs the root node of a graph");
  if (root->kind != HPVM_NODE_INTERNAL || root->ndims != 0)
    return fail(HPVM_ERR_INVALID_GRAPH, "the root must be a single-instance internal node");
  if (!args || args_size < kRecBytes)
    return fail(HPVM_ERR_INVALID_ARG, "argument record too small (%zu < %zu bytes)", args_size, kRecBytes);
  int rc = validated ? HPVM_OK : validate_node(root);
  if (rc != HPVM_OK) return rc;
  P->R = Records{static_cast<const uint8_t*>(args), (int)std::min<size_t>(args_size / kRecBytes, kMaxRecords)};
  std::vector<hpvm_node*> order;
  if ((rc = topo_children(root, &order)) != HPVM_OK) return rc;
  if (order.empty()) return fail(HPVM_ERR_UNSUPPORTED, "the root holds no tile node");
  for (auto* st : order)
    if (st->kind != HPVM_NODE_INTERNAL || st->ndims != 2)
      return fail(HPVM_ERR_UNSUPPORTED, "every child of the root must be a 2-D internal node (a tile grid)");
  for (auto* e : root->edges)
    if (e->repl != HPVM_ALL_TO_ALL)
      return fail(HPVM_ERR_UNSUPPORTED,
                  "edges between tile grids must be all-to-all (a whole result feeds the next stage)");
  P->stages.clear();
  for (auto* st : order) {
    Stage S;
    if ((rc = lower_stage(st, P->R, &S)) != HPVM_OK) return rc;
    P->stages.push_back(S);
  }
  return HPVM_OK;
}

int32_t record_i32(const Plan& P, int rec, size_t off) {
  int32_t v;
  memcpy(&v, P.R.base + rec * kRecBytes + off, 4);
  return v;
}

int check_stage_tier(const Stage& S, int tier) {
  if (tier < HPVM_TIER_FP32_DFG || tier > HPVM_TIER_BF16X6) return fail(HPVM_ERR_INVALID_ARG, "unknown tier %d", tier);
  if (tier == HPVM_TIER_FP32_DFG) {
    if (S.block_x != S.block_y)
      return fail(HPVM_ERR_UNSUPPORTED, "the FP32_DFG lowering needs a square leaf grid (got %lld x %lld)",
                  (long long)S.block_x, (long long)S.block_y);
    if (S.block_x * S.block_y > 1024)
      return fail(HPVM_ERR_UNSUPPORTED, "the FP32_DFG lowering maps leaf instances to threads: at most 1024");
    if (!S.has_a_tile)
      return fail(HPVM_ERR_UNSUPPORTED, "the FP32_DFG lowering needs the Allocation's A tile (ports 14, 15)");
    if (S.alloc_bx * S.alloc_by < S.block_x * S.block_y)
      return fail(HPVM_ERR_SHAPE, "the Allocation tile (%lld x %lld) is smaller than the leaf grid",
                  (long long)S.alloc_bx, (long long)S.alloc_by);
  }
  return HPVM_OK;
}

size_t workspace_need(const Stage& S, int tier) {
  if (tier == HPVM_TIER_BF16X3 || tier == HPVM_TIER_BF16 || tier == HPVM_TIER_FP8 || tier == HPVM_TIER_BF16X6)
    return hpvm::tc_workspace_bytes(S.d, tier);
  return 0;
}

// Streaming edges lowered into the producer's epilogue: stage i's result C
// is stage i+1's op(B) = B (K of stage i+1 = M of stage i) on the same
// BF16x3 or BF16 tier, merged (no HPVM_LAUNCH_NO_FUSION) and not taken from
// the plane cache. Stage i's epilogue then also writes the planes of C that
// stage i+1 reads, and stage i+1 skips its conversion of B: the result makes
// one trip through HBM instead of being written, read back and converted.
bool forwards_b(const Plan& P, size_t i) {
  if (i + 1 >= P.stages.size()) return false;
  const Stage& a = P.stages[i];
  const Stage& b = P.stages[i + 1];
  const int tier = record_i32(P, a.rec, kTierOffset);
  if (tier != record_i32(P, b.rec, kTierOffset) || (tier != HPVM_TIER_BF16X3 && tier != HPVM_TIER_BF16))
    return false;
  const int fa = record_i32(P, a.rec, kFlagsOffset), fb = record_i32(P, b.rec, kFlagsOffset);
  if ((fa | fb) & HPVM_LAUNCH_NO_FUSION) return false;
  if (fb & (HPVM_LAUNCH_CACHE_B | HPVM_LAUNCH_REUSE_B)) return false;
  const hpvm::SgemmDesc& x = a.d;
  const hpvm::SgemmDesc& y = b.d;
  return x.M > 0 && x.N > 0 && y.M > 0 && y.K > 0 && y.B == x.C && !y.transB && y.ldb == x.ldc &&
         y.K == x.M && y.N == x.N;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace of a plan: the planes of its largest stage, then (when stages
// forward planes) two regions for forwarded planes, used alternately so a
// stage reads its B from one while its epilogue writes the next stage's
// into the other.
struct WsPlan {
  size_t stage = 0, fwd = 0;
  size_t total() const { return fwd ? align256(stage) + 2 * align256(fwd) : stage; }
  size_t region(size_t i) const { return align256(stage) + (i & 1) * align256(fwd); }
};
WsPlan plan_ws(const Plan& P) {
  WsPlan W;
  for (size_t i = 0; i < P.stages.size(); ++i) {
    const Stage& S = P.stages[i];
    const int tier = record_i32(P, S.rec, kTierOffset);
    W.stage = std::max(W.stage, workspace_need(S, tier));
    if (forwards_b(P, i)) W.fwd = std::max(W.fwd, hpvm::tc_operand_layout(tier, S.d.N, S.d.M).total);
  }
  return W;
}

size_t plan_workspace(const Plan& P) { return plan_ws(P).total(); }

TrackEntry* find_tracked(hpvm_ctx* ctx, const void* p, int64_t* offset) {
  const char* c = static_cast<const char*>(p);
  for (auto& t : ctx->tracked)
    if (c >= t.host && c < t.host + std::max<int64_t>(t.bytes, 1)) {
      *offset = c - t.host;
      return &t;
    }
  return nullptr;
}

int check_device_pointer(const void* p, const char* name) {
  if (!p) return HPVM_OK;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(HPVM_ERR_INVALID_ARG, "%s is neither device memory nor a tracked host region", name);
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(HPVM_ERR_INVALID_ARG, "%s is host memory that was not registered with hpvm_track_mem", name);
  return HPVM_OK;
}

// Map a record pointer to the device: tracked host regions use their device
// copy (copied in first when `read` and the device copy is stale).
int map_pointer(hpvm_ctx* ctx, const void* p, bool read, cudaStream_t s, const char* name, void** out,
                TrackEntry** entry, int64_t* h2d) {
  *entry = nullptr;
  *out = const_cast<void*>(p);
  if (!p) return HPVM_OK;
  int64_t off = 0;
  TrackEntry* t = find_tracked(ctx, p, &off);
  if (!t) return check_device_pointer(p, name);
  if (!t->dev) {
    cudaError_t e = cudaMalloc(&t->dev, (size_t)std::max<int64_t>(t->bytes, 1));
    if (e != cudaSuccess) {
      t->dev = nullptr;
      return fail(HPVM_ERR_OUT_OF_MEMORY, "device copy of a tracked region (%lld bytes): %s", (long long)t->bytes,
                  cudaGetErrorString(e));
    }
    t->dev_valid = false;
  }
  if (read && !t->dev_valid) {
    cudaError_t e = cudaMemcpyAsync(t->dev, t->host, (size_t)t->bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "host->device copy of a tracked region");
    t->dev_valid = true;
    *h2d += t->bytes;
  }
  *entry = t;
  *out = static_cast<char*>(t->dev) + off;
  return HPVM_OK;
}

// Records on s that the launch enqueued so far wrote t's device copy, so
// that request_mem waits for that launch alone. Inside a stream capture no
// event is recorded and request_mem falls back to waiting for the device.
int mark_written(TrackEntry* t, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    t->written_set = false;
    return HPVM_OK;
  }
  cudaError_t e = cudaSuccess;
  if (!t->written) e = cudaEventCreateWithFlags(&t->written, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(t->written, s);
  if (e != cudaSuccess) return cuda_fail(e, "recording the write of a tracked region");
  t->written_set = true;
  return HPVM_OK;
}

int grow_buffer(void** buf, size_t* have, size_t need, cudaStream_t sync_on) {
  if (need == 0 || (*buf && *have >= need)) return HPVM_OK;
  if (*buf) {
    if (sync_on) cudaStreamSynchronize(sync_on);
    else cudaDeviceSynchronize();
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
  }
  cudaError_t e = cudaMalloc(buf, need);
  if (e != cudaSuccess) {
    *buf = nullptr;
    return fail(HPVM_ERR_OUT_OF_MEMORY, "workspace of %zu bytes: %s", need, cudaGetErrorString(e));
  }
  *have = need;
  return HPVM_OK;
}

int ensure_workspace(hpvm_ctx* ctx, size_t need, void** ws, size_t* ws_bytes) {
  if (need == 0 || (ctx->ws && ctx->ws_bytes >= need)) {
    *ws = ctx->ws;
    *ws_bytes = ctx->ws_bytes;
    return HPVM_OK;
  }
  if (ctx->ws && !ctx->ws_owned)
    return fail(HPVM_ERR_SHAPE, "the workspace set with hpvm_set_workspace has %zu bytes, this launch needs %zu",
                ctx->ws_bytes, need);
  int rc = grow_buffer(&ctx->ws, &ctx->ws_bytes, need, nullptr);
  if (rc != HPVM_OK) return rc;
  ctx->ws_owned = true;
  *ws = ctx->ws;
  *ws_bytes = ctx->ws_bytes;
  return HPVM_OK;
}

// Enqueue every stage of a lowered graph on stream s.
// Waits for every launch that reads a cached plane, then frees the cache.
void free_planes(hpvm_ctx* ctx) {
  for (auto& e : ctx->planes) {
    for (auto& u : e->uses) {
      cudaEventSynchronize(u.second);
      cudaEventDestroy(u.second);
    }
    if (e->converted) {
      cudaEventSynchronize(e->converted);
      cudaEventDestroy(e->converted);
    }
    if (e->buf) cudaFree(e->buf);
  }
  ctx->planes.clear();
  ctx->plane_bytes = 0;
}

// The plane cache entry of an operand (key: its device pointer, leading
// dimension, rows, K, source layout and tier) and what the leaf does with
// it: read its planes (reuse of a valid entry; on another stream only after
// the event of its conversion) or convert into them (a refill waits for the
// launches on other streams that still read them). *out stays null when the
// cache has no room: the operand is then converted into the workspace.
int plane_entry(hpvm_ctx* ctx, const void* src, int64_t ld, int64_t rows, int64_t K, int layout, int tier,
                bool reuse, cudaStream_t s, PlaneEntry** out, hpvm::OperandPlanes* op) {
  *out = nullptr;
  *op = hpvm::OperandPlanes();
  PlaneEntry* e = nullptr;
  for (auto& p : ctx->planes)
    if (p->src == src && p->ld == ld && p->rows == rows && p->K == K && p->layout == layout && p->tier == tier) {
      e = p.get();
      break;
    }
  if (!e) {
    const size_t bytes = hpvm::tc_operand_layout(tier, rows, K).total;
    if (ctx->plane_bytes + bytes > kPlaneCacheLimit) return HPVM_OK;
    auto ne = std::make_unique<PlaneEntry>();
    ne->src = src;
    ne->ld = ld;
    ne->rows = rows;
    ne->K = K;
    ne->layout = layout;
    ne->tier = tier;
    if (cudaMalloc(&ne->buf, bytes) != cudaSuccess) {
      cudaGetLastError();  // no room on the device: convert into the workspace
      return HPVM_OK;
    }
    cudaError_t c = cudaEventCreateWithFlags(&ne->converted, cudaEventDisableTiming);
    if (c != cudaSuccess) {
      cudaFree(ne->buf);
      return cuda_fail(c, "cudaEventCreate");
    }
    ne->bytes = bytes;
    ctx->plane_bytes += bytes;
    e = ne.get();
    ctx->planes.push_back(std::move(ne));
  }
  op->base = e->buf;
  if (reuse && e->valid) {
    if (e->filled_on != s) cudaStreamWaitEvent(s, e->converted, 0);
    op->ready = true;
  } else {
    for (auto& u : e->uses)
      if (u.first != s) cudaStreamWaitEvent(s, u.second, 0);
    e->valid = false;
    op->converted = e->converted;
  }
  *out = e;
  return HPVM_OK;
}

// Marks every cache entry of src read with this leading dimension, rows, K
// and layout (any tier) as not holding the operand: its next use converts.
void invalidate_planes(hpvm_ctx* ctx, const void* src, int64_t ld, int64_t rows, int64_t K, int layout) {
  for (auto& p : ctx->planes)
    if (p->src == src && p->ld == ld && p->rows == rows && p->K == K && p->layout == layout) p->valid = false;
}

// After a launch on stream s read (or filled) entry e.
int plane_used(PlaneEntry* e, const hpvm::OperandPlanes& op, cudaStream_t s) {
  if (!op.ready) {
    e->valid = true;
    e->filled_on = s;
  }
  for (auto& u : e->uses)
    if (u.first == s) {
      cudaError_t c = cudaEventRecord(u.second, s);
      return c == cudaSuccess ? HPVM_OK : cuda_fail(c, "cudaEventRecord");
    }
  cudaEvent_t ev;
  cudaError_t c = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (c == cudaSuccess) c = cudaEventRecord(ev, s);
  if (c != cudaSuccess) return cuda_fail(c, "plane cache event");
  e->uses.emplace_back(s, ev);
  return HPVM_OK;
}

int execute_plan(hpvm_ctx* ctx, const Plan& P, cudaStream_t s, void* ws, size_t ws_bytes, hpvm_launch_info* inf) {
  memset(inf, 0, sizeof *inf);
  int64_t h2d = 0;
  int rc;
  bool first = true;
  const WsPlan WP = plan_ws(P);
  if (WP.fwd && (!ws || ws_bytes < WP.total()))
    return fail(HPVM_ERR_SHAPE, "workspace of %zu bytes, the plan needs %zu", ws_bytes, WP.total());
  for (size_t si = 0; si < P.stages.size(); ++si) {
    const Stage& S0 = P.stages[si];
    const int tier = record_i32(P, S0.rec, kTierOffset);
    const int flags = record_i32(P, S0.rec, kFlagsOffset);
    if ((rc = check_stage_tier(S0, tier)) != HPVM_OK) return rc;
    Stage S = S0;
    const bool work = S.d.M > 0 && S.d.N > 0;
    void *A = nullptr, *B = nullptr, *C = nullptr, *H = nullptr;
    TrackEntry *tA = nullptr, *tB = nullptr, *tC = nullptr, *tH = nullptr;
    if (work && S.d.K > 0) {
      if ((rc = map_pointer(ctx, S.d.A, true, s, "A", &A, &tA, &h2d)) != HPVM_OK) return rc;
      if ((rc = map_pointer(ctx, S.d.B, true, s, "B", &B, &tB, &h2d)) != HPVM_OK) return rc;
    }
    if (work) {
      if ((rc = map_pointer(ctx, S.d.C, S.d.beta != 0.f, s, "C", &C, &tC, &h2d)) != HPVM_OK) return rc;
      if (S.epi.kind == 2 && (rc = map_pointer(ctx, S.epi.aux, true, s, "H", &H, &tH, &h2d)) != HPVM_OK) return rc;
    }
    S.d.A = static_cast<const float*>(A);
    S.d.B = static_cast<const float*>(B);
    S.d.C = static_cast<float*>(C);
    if (S.epi.kind == 2) S.epi.aux = static_cast<const float*>(H);
    hpvm::KernelReport rep;
    if (work) {
      std::string err;
      hpvm::LaunchHooks hooks;
      if (ctx->timing) {
        if (cudaEventCreate(&hooks.main_begin) != cudaSuccess || cudaEventCreate(&hooks.main_end) != cudaSuccess)
          return fail(HPVM_ERR_CUDA, "cannot create timing events");
        ctx->timed.emplace_back(hooks.main_begin, hooks.main_end);
      }
      // MergeDependentNodes: the tensor-core leaves take the elementwise
      // leaf into their epilogue; the FP32 leaves, the BF16X6 leaf (built
      // with the plain epilogue only) and HPVM_LAUNCH_NO_FUSION run it as
      // its own kernel after the sgemm leaf.
      const bool tensor = tier >= HPVM_TIER_BF16X3;
      const bool fuse = tensor && tier != HPVM_TIER_BF16X6 && !(flags & HPVM_LAUNCH_NO_FUSION);
      // operand plane cache (A's rows are contiguous unless transposed, B's
      // N rows only when transposed: the layouts the conversions read)
      hpvm::OperandPlanes pa, pb;
      PlaneEntry *ea = nullptr, *eb = nullptr;
      if (tensor && S.d.K > 0) {
        if ((flags & (HPVM_LAUNCH_CACHE_A | HPVM_LAUNCH_REUSE_A)) &&
            (rc = plane_entry(ctx, S.d.A, S.d.lda, S.d.M, S.d.K, !S.d.transA, tier,
                              !(flags & HPVM_LAUNCH_CACHE_A), s, &ea, &pa)) != HPVM_OK)
          return rc;
        if ((flags & (HPVM_LAUNCH_CACHE_B | HPVM_LAUNCH_REUSE_B)) &&
            (rc = plane_entry(ctx, S.d.B, S.d.ldb, S.d.N, S.d.K, S.d.transB != 0, tier,
                              !(flags & HPVM_LAUNCH_CACHE_B), s, &eb, &pb)) != HPVM_OK)
          return rc;
        if (ea && ea == eb) {
          // one entry serves both operands (the same matrix): A's conversion,
          // which the leaf launch runs first, fills it for both
          pb = pa;
          pb.ready = true;
          pb.converted = nullptr;
          eb = nullptr;
        }
        if (si > 0 && forwards_b(P, si - 1)) {
          // B's planes were written by the previous stage's epilogue
          pb = hpvm::OperandPlanes();
          pb.base = static_cast<uint8_t*>(ws) + WP.region(si - 1);
          pb.ready = true;
        }
      }
      if (forwards_b(P, si)) S.epi.fwd = static_cast<uint8_t*>(ws) + WP.region(si);
      // HPVM_LAUNCH_CACHE_C: the merged elementwise leaf's epilogue fills
      // the cache entry of C read with C's rows as operand rows (the key of
      // op(A) = A or op(B) = B^T over C, K = N); a stage that cannot (no
      // merged leaf, FP8) drops the entry's contents instead
      hpvm::OperandPlanes pc;
      PlaneEntry* ec = nullptr;
      if (flags & HPVM_LAUNCH_CACHE_C) {
        if (fuse && S.epi.kind != 0 && (tier == HPVM_TIER_BF16 || tier == HPVM_TIER_BF16X3)) {
          if ((rc = plane_entry(ctx, S.d.C, S.d.ldc, S.d.M, S.d.N, 1, tier, false, s, &ec, &pc)) != HPVM_OK)
            return rc;
          if (ec) S.epi.rows = pc.base;
        } else {
          invalidate_planes(ctx, S.d.C, S.d.ldc, S.d.M, S.d.N, 1);
        }
      }
      // HPVM_LAUNCH_PLANES_ONLY: C is read only through the planes this
      // stage writes, so the FP32 C is not stored. Honoured only where those
      // planes exist for every reader the flags name (forwarded to the next
      // stage, and the cache entry when CACHE_C asked for one), with beta = 0
      // and C not a tracked host region; otherwise C is stored as usual.
      if ((flags & HPVM_LAUNCH_PLANES_ONLY) && fuse && S.d.beta == 0.f && !tC && (S.epi.fwd || S.epi.rows) &&
          (!(flags & HPVM_LAUNCH_CACHE_C) || S.epi.rows))
        S.epi.planes_only = true;
      hpvm::Epilogue none;
      none.split_as = S.epi.kind;  // unmerged: split the tail as the merged leaf would
      S.epi.separate_split = none.separate_split = (flags & HPVM_LAUNCH_SEPARATE_SPLIT) != 0;
      cudaError_t e;
      switch (tier) {
        case HPVM_TIER_FP32_DFG:
          e = hpvm::launch_fp32_dfg(S.d, (int)S.block_x, (int)S.grid_x, (int)S.grid_y,
                                    (size_t)(S.block_x * S.block_y * 4), s, &rep, &hooks);
          break;
        case HPVM_TIER_FP32:
          e = hpvm::launch_fp32_tiled(S.d, s, &rep, &hooks);
          break;
        default:
          e = hpvm::launch_tc(S.d, tier, ws, ws_bytes, ctx->status, s, &rep, &err, &hooks, fuse ? S.epi : none,
                              pa, pb);
          if (e == cudaErrorInvalidValue && !err.empty()) return fail(HPVM_ERR_SHAPE, "%s", err.c_str());
          break;
      }
      if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
      if (ea && (rc = plane_used(ea, pa, s)) != HPVM_OK) return rc;
      if (eb && (rc = plane_used(eb, pb, s)) != HPVM_OK) return rc;
      if (ec) {
        if ((e = cudaEventRecord(ec->converted, s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
        if ((rc = plane_used(ec, pc, s)) != HPVM_OK) return rc;
      }
      if (S.epi.kind && !fuse) {
        e = hpvm::launch_elementwise(S.d, S.epi, s);
        if (e != cudaSuccess) return cuda_fail(e, "elementwise leaf launch");
        rep.kernels += 1;
      }
    }
    if (tC) {
      tC->dev_valid = true;
      tC->host_valid = false;
      if ((rc = mark_written(tC, s)) != HPVM_OK) return rc;
    }
    if (first) {  // the first stage describes the launch
      inf->tier = tier;
      inf->grid_x = rep.grid_x;
      inf->grid_y = rep.grid_y;
      inf->grid_z = rep.grid_z;
      inf->block_threads = rep.block_threads;
      inf->tile_m = rep.tile_m;
      inf->tile_n = rep.tile_n;
      inf->tile_k = rep.tile_k;
      inf->smem_bytes = rep.smem_bytes;
      inf->literal = rep.literal;
      first = false;
    }
    inf->kernels += rep.kernels;
    inf->workspace_bytes = std::max<int64_t>(inf->workspace_bytes, rep.workspace_bytes);
  }
  inf->h2d_bytes = h2d;
  return HPVM_OK;
}

int wait_event(cudaEvent_t ev, int64_t timeout_ms) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return HPVM_OK;
    if (e != cudaErrorNotReady) return cuda_fail(e, "waiting for the graph");
    if (timeout_ms >= 0 && std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
      return fail(HPVM_ERR_TIMEOUT, "graph not finished after %lld ms", (long long)timeout_ms);
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

int check_status(hpvm_ctx* ctx) {
  if (!ctx->status.host) return HPVM_OK;
  int st = *const_cast<volatile int*>(ctx->status.host);
  if (st) {
    *const_cast<volatile int*>(ctx->status.host) = 0;
    return fail(HPVM_ERR_DEVICE_FAULT, "a kernel gave up a bounded wait (status bits 0x%x)", st);
  }
  return HPVM_OK;
}

// ---- streaming: items run one launch each, or several as one launch ----------
cudaEvent_t take_event(hpvm_graph* g) {
  cudaEvent_t ev = nullptr;
  if (!g->spare_events.empty()) {
    ev = g->spare_events.back();
    g->spare_events.pop_back();
  } else if (!g->ctx->spare_events.empty()) {
    ev = g->ctx->spare_events.back();
    g->ctx->spare_events.pop_back();
  } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    ev = nullptr;
  }
  return ev;
}

// One item on the next stream of the ring.
int launch_item(hpvm_graph* g, StreamItem& it) {
  hpvm_ctx* ctx = g->ctx;
  Plan P;
  int rc = lower_graph(g->root, it.record.data(), it.record.size(), &P, g->validated == ctx->structure);
  if (rc != HPVM_OK) return rc;
  const int slot = (int)(g->launches % g->slots.size());
  cudaStream_t s = g->slots[slot];
  if ((rc = grow_buffer(&g->slot_ws[slot], &g->slot_ws_bytes[slot], plan_workspace(P), s)) != HPVM_OK) return rc;
  hpvm_launch_info inf;
  if ((rc = execute_plan(ctx, P, s, g->slot_ws[slot], g->slot_ws_bytes[slot], &inf)) != HPVM_OK) return rc;
  if (!it.done && !(it.done = take_event(g))) return fail(HPVM_ERR_CUDA, "cudaEventCreate failed");
  cudaEventRecord(it.done, s);
  it.launched = true;
  g->info = inf;
  g->launches++;
  return HPVM_OK;
}

// Whether items can run as one launch: the same records but for stage 0's
// B (each item's own, K x N_j column-major with ldb = K, op(B) = B), the
// last stage's C (each item's own, ldc = M) and the items' N; every stage
// with beta = 0 (C is not read) and no auxiliary matrix, every pointer on
// the device; the plane-cache flags may differ only in CACHE_A / REUSE_A
// (the items share A: the group converts it if any item asks for it), and
// none may cache B or C. Then the stages run once over N = sum N_j: the items' B
// operands copied side by side into one matrix, every stage's result into
// one matrix (two alternating), the last one copied back out to the
// items' C.
bool coalescible(hpvm_ctx* ctx, const std::vector<StreamItem*>& batch, int nrec) {
  using R = hpvm_sgemm_root_args;
  if (batch.size() < 2 || nrec < 1) return false;
  const R* r0 = reinterpret_cast<const R*>(batch[0]->record.data());
  for (auto* it : batch) {
    if ((int)(it->record.size() / sizeof(R)) != nrec) return false;
    const R* r = reinterpret_cast<const R*>(it->record.data());
    for (int l = 0; l < nrec; ++l) {
      const R& a = r0[l];
      const R& b = r[l];
      if (b.beta != 0.f || b.aux || b.A != a.A || b.lda != a.lda || b.M != a.M || b.k != a.k ||
          b.transA != a.transA || b.transB != a.transB || b.tier != a.tier ||
          ((b.flags ^ a.flags) & ~(HPVM_LAUNCH_CACHE_A | HPVM_LAUNCH_REUSE_A)) ||
          (b.flags & (HPVM_LAUNCH_CACHE_B | HPVM_LAUNCH_REUSE_B | HPVM_LAUNCH_CACHE_C)) ||
          b.alpha != a.alpha || b.block_x != a.block_x || b.block_y != a.block_y || b.grid_x != a.grid_x ||
          b.N != r[0].N || b.N <= 0 || b.ldc != b.M || !b.C)
        return false;
      if (l > 0 && b.B) return false;  // later stages read the previous stage's result
      int64_t off;
      if (find_tracked(ctx, b.C, &off)) return false;
    }
    int64_t off;
    if (!r[0].B || r[0].transB || r[0].ldb != r[0].k || find_tracked(ctx, r[0].B, &off)) return false;
  }
  return true;
}

int launch_coalesced(hpvm_graph* g, std::vector<StreamItem*>& batch) {
  using R = hpvm_sgemm_root_args;
  hpvm_ctx* ctx = g->ctx;
  const int nrec = (int)(batch[0]->record.size() / sizeof(R));
  std::vector<R> rec(nrec);
  memcpy(rec.data(), batch[0]->record.data(), nrec * sizeof(R));
  for (int l = 0; l < nrec; ++l)  // A converted into the cache if any item asks for it
    for (auto* it : batch)
      if (reinterpret_cast<const R*>(it->record.data())[l].flags & HPVM_LAUNCH_CACHE_A) {
        rec[l].flags = (rec[l].flags & ~HPVM_LAUNCH_REUSE_A) | HPVM_LAUNCH_CACHE_A;
        break;
      }
  std::vector<int64_t> off(batch.size() + 1, 0);
  for (size_t j = 0; j < batch.size(); ++j)
    off[j + 1] = off[j] + reinterpret_cast<const R*>(batch[j]->record.data())[0].N;
  const int64_t N = off.back();
  const int64_t K0 = rec[0].k;
  int64_t Mmax = 0;
  for (auto& r : rec) Mmax = std::max<int64_t>(Mmax, r.M);
  // The items' first operands, or their last results, that already lie side
  // by side in memory (say views of one batch tensor) are used in place;
  // otherwise they are gathered into (returned from) the workspace.
  auto adjacent = [&](int l, bool c) {
    const float* base = c ? reinterpret_cast<const R*>(batch[0]->record.data())[l].C
                          : reinterpret_cast<const R*>(batch[0]->record.data())[l].B;
    const int64_t ld = c ? rec[l].M : K0;
    for (size_t j = 1; j < batch.size(); ++j) {
      const R& r = reinterpret_cast<const R*>(batch[j]->record.data())[l];
      if ((c ? r.C : r.B) != base + off[j] * ld) return false;
    }
    return true;
  };
  const bool b_in_place = adjacent(0, false), c_in_place = adjacent(nrec - 1, true);
  const size_t xbytes = b_in_place ? 0 : align256((size_t)K0 * N * 4), cbytes = align256((size_t)Mmax * N * 4);
  // the combined records: N summed, the tile grid along N to match, stage
  // 0's B and every stage's C in the scratch matrices (pointers set once the
  // workspace is placed)
  auto fill = [&](uint8_t* scratch) {
    for (int l = 0; l < nrec; ++l) {
      R& r = rec[l];
      r.N = (int32_t)N;
      r.grid_y = (int32_t)((N + r.block_y - 1) / r.block_y);
      r.C = reinterpret_cast<float*>(scratch + xbytes + (l & 1) * cbytes);
      r.bytesC = (int64_t)r.M * N * 4;
    }
    if (c_in_place) rec[nrec - 1].C = reinterpret_cast<const R*>(batch[0]->record.data())[nrec - 1].C;
    rec[0].B = b_in_place ? reinterpret_cast<const R*>(batch[0]->record.data())[0].B
                          : reinterpret_cast<float*>(scratch);
    rec[0].bytesB = K0 * N * 4;
  };
  fill(reinterpret_cast<uint8_t*>(uintptr_t(256)));
  Plan P;
  int rc = lower_graph(g->root, rec.data(), nrec * sizeof(R), &P, g->validated == ctx->structure);
  if (rc != HPVM_OK) return rc;
  const size_t wsb = align256(plan_workspace(P));
  const int slot = (int)(g->launches % g->slots.size());
  cudaStream_t s = g->slots[slot];
  if ((rc = grow_buffer(&g->slot_ws[slot], &g->slot_ws_bytes[slot], wsb + xbytes + 2 * cbytes, s)) != HPVM_OK)
    return rc;
  uint8_t* scratch = static_cast<uint8_t*>(g->slot_ws[slot]) + wsb;
  fill(scratch);
  if ((rc = lower_graph(g->root, rec.data(), nrec * sizeof(R), &P, true)) != HPVM_OK) return rc;
  cudaError_t e;
  for (size_t j = 0; j < batch.size() && !b_in_place; ++j) {
    const R& r = reinterpret_cast<const R*>(batch[j]->record.data())[0];
    if ((e = cudaMemcpyAsync(scratch + off[j] * K0 * 4, r.B, (size_t)(off[j + 1] - off[j]) * K0 * 4,
                             cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "gathering the items' operands");
  }
  hpvm_launch_info inf;
  if ((rc = execute_plan(ctx, P, s, g->slot_ws[slot], wsb, &inf)) != HPVM_OK) return rc;
  const R& last = rec[nrec - 1];
  for (size_t j = 0; j < batch.size() && !c_in_place; ++j) {
    const R& r = reinterpret_cast<const R*>(batch[j]->record.data())[nrec - 1];
    if ((e = cudaMemcpyAsync(r.C, reinterpret_cast<const uint8_t*>(last.C) + off[j] * last.M * 4,
                             (size_t)(off[j + 1] - off[j]) * last.M * 4, cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
      return cuda_fail(e, "returning the items' results");
  }
  for (auto* it : batch) {
    if (!it->done && !(it->done = take_event(g))) return fail(HPVM_ERR_CUDA, "cudaEventCreate failed");
    cudaEventRecord(it->done, s);
    it->launched = true;
  }
  g->info = inf;
  g->launches++;
  return HPVM_OK;
}

// Launch every queued item: groups of up to g->coalesce items that can run
// as one launch do, the others one by one.
int flush_items(hpvm_graph* g) {
  std::vector<StreamItem*> waiting;
  for (auto& it : g->items)
    if (!it.launched) waiting.push_back(&it);
  size_t i = 0;
  while (i < waiting.size()) {
    const size_t n = std::min<size_t>(waiting.size() - i, (size_t)std::max(1, g->coalesce));
    std::vector<StreamItem*> batch(waiting.begin() + i, waiting.begin() + i + n);
    int rc;
    const int nrec = (int)(batch[0]->record.size() / sizeof(hpvm_sgemm_root_args));
    if (n > 1 && coalescible(g->ctx, batch, nrec)) {
      rc = launch_coalesced(g, batch);
    } else {
      rc = HPVM_OK;
      for (auto* it : batch)
        if ((rc = launch_item(g, *it)) != HPVM_OK) break;
    }
    if (rc != HPVM_OK) return rc;
    i += n;
  }
  return HPVM_OK;
}

// keep: hand the streams, slot workspaces and events to the context for
// the next streaming graph (after the graph's work is done); otherwise
// destroy them
void free_graph(hpvm_graph* g, bool keep = false) {
  hpvm_ctx* ctx = g->ctx;
  if (g->done) cudaEventDestroy(g->done);
  for (auto& it : g->items)
    if (it.done) cudaEventDestroy(it.done);
  for (auto ev : g->spare_events) {
    if (keep) ctx->spare_events.push_back(ev);
    else cudaEventDestroy(ev);
  }
  // (last slot first: the next graph, taking them from the back, gets each
  // slot's workspace back in the same slot, sized for the same work)
  for (size_t i = g->slots.size(); i-- > 0;) {
    if (g->slots[i]) {
      cudaStreamSynchronize(g->slots[i]);
      if (keep) ctx->spare_streams.push_back(g->slots[i]);
      else cudaStreamDestroy(g->slots[i]);
    }
    if (g->slot_ws[i]) {
      if (keep) ctx->spare_ws.emplace_back(g->slot_ws[i], g->slot_ws_bytes[i]);
      else cudaFree(g->slot_ws[i]);
    }
  }
  delete g;
}

}  // namespace

// ===========================================================================
// C-ABI
extern "C" {

const char* hpvm_last_error(void) { return g_last_error.c_str(); }
int hpvm_version(void) { return 201; }

int hpvm_init(int device, hpvm_ctx** out) {
  if (!out) return fail(HPVM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  auto ctx = std::make_unique<hpvm_ctx>();
  ctx->device = device;
  if (device >= 0) {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device >= n) {
      cudaGetLastError();
      return fail(HPVM_ERR_NO_DEVICE, "CUDA device %d is not available", device);
    }
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    int* h = nullptr;
    e = cudaHostAlloc(reinterpret_cast<void**>(&h), sizeof(int), cudaHostAllocMapped);
    if (e != cudaSuccess) return cuda_fail(e, "status word");
    *h = 0;
    int* dptr = nullptr;
    e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&dptr), h, 0);
    if (e != cudaSuccess) {
      cudaFreeHost(h);
      return cuda_fail(e, "status word device address");
    }
    ctx->status.host = h;
    ctx->status.dev = dptr;
  }
  *out = ctx.release();
  return ok();
}

int hpvm_cleanup(hpvm_ctx* ctx) {
  if (!ctx) return fail(HPVM_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->device >= 0) {
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto* g : ctx->graphs) free_graph(g);
    for (auto& t : ctx->tracked) {
      if (t.dev) cudaFree(t.dev);
      if (t.written) cudaEventDestroy(t.written);
    }
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (auto st : ctx->spare_streams) cudaStreamDestroy(st);
    for (auto& w : ctx->spare_ws) cudaFree(w.first);
    for (auto ev : ctx->spare_events) cudaEventDestroy(ev);
    if (ctx->ws && ctx->ws_owned) cudaFree(ctx->ws);
    if (ctx->ws_event) cudaEventDestroy(ctx->ws_event);
    if (ctx->status.host) cudaFreeHost(ctx->status.host);
    for (auto& pr : ctx->timed) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    for (auto* b : ctx->batches) {
      hpvm::tc_batch_free(&b->tb);
      delete b;
    }
    free_planes(ctx);
  }
  delete ctx;
  return ok();
}

int hpvm_create_node(hpvm_ctx* ctx, hpvm_node* parent, int kind, int ndims, const int64_t* dims,
                     hpvm_node** out) {
  if (!ctx || !out) return fail(HPVM_ERR_INVALID_ARG, "ctx or out is NULL");
  *out = nullptr;
  if (kind < HPVM_NODE_INTERNAL || kind > HPVM_NODE_TANH_GRAD_LEAF)
    return fail(HPVM_ERR_INVALID_ARG, "unknown node kind %d", kind);
  if (ndims < 0 || ndims > 3) return fail(HPVM_ERR_INVALID_ARG, "ndims must be 0..3, got %d", ndims);
  if (ndims > 0 && !dims) return fail(HPVM_ERR_INVALID_ARG, "dims is NULL");
  if (parent) {
    if (parent->ctx != ctx) return fail(HPVM_ERR_INVALID_ARG, "parent belongs to another context");
    if (is_leaf(parent))
      return fail(HPVM_ERR_INVALID_GRAPH, "%s is a leaf: only internal nodes hold child graphs",
                  node_label(parent).c_str());
  } else if (kind != HPVM_NODE_INTERNAL || ndims != 0) {
    return fail(HPVM_ERR_INVALID_GRAPH, "a root node must be a single-instance internal node");
  }
  auto n = std::make_unique<hpvm_node>();
  n->ctx = ctx;
  n->parent = parent;
  n->kind = kind;
  n->ndims = ndims;
  for (int d = 0; d < ndims; ++d) {
    if (dims[d] == 0) return fail(HPVM_ERR_INVALID_ARG, "extent %d is 0", d);
    if (dims[d] < 0) {
      int64_t p = -1 - dims[d];
      if (!parent || p >= in_arity(parent))
        return fail(HPVM_ERR_INVALID_ARG, "extent %d names parent input %lld, out of range", d, (long long)p);
    }
    n->dims[d] = dims[d];
  }
  n->id = ctx->next_id++;
  hpvm_node* raw = n.get();
  ctx->nodes.push_back(std::move(n));
  if (parent) parent->children.push_back(raw);
  ctx->structure++;
  *out = raw;
  return ok();
}

int hpvm_create_edge(hpvm_node* src, hpvm_node* dst, int repl, int sp, int dp, int stream, hpvm_edge** out) {
  if (out) *out = nullptr;
  if (!src || !dst) return fail(HPVM_ERR_INVALID_ARG, "src or dst is NULL");
  if (repl != HPVM_ONE_TO_ONE && repl != HPVM_ALL_TO_ALL)
    return fail(HPVM_ERR_INVALID_ARG, "replication type must be one-to-one (0) or all-to-all (1)");
  if (src == dst) return fail(HPVM_ERR_INVALID_GRAPH, "an edge from a node to itself");
  if (!src->parent || src->parent != dst->parent)
    return fail(HPVM_ERR_INVALID_GRAPH, "an edge must join two children of the same internal node");
  if (sp < 0 || sp >= out_arity(src))
    return fail(HPVM_ERR_INVALID_ARG, "output %d of %s is out of range", sp, node_label(src).c_str());
  if (dp < 0 || dp >= in_arity(dst))
    return fail(HPVM_ERR_INVALID_ARG, "input %d of %s is out of range", dp, node_label(dst).c_str());
  if (repl == HPVM_ONE_TO_ONE) {
    bool same = src->ndims == dst->ndims;
    for (int d = 0; same && d < src->ndims; ++d) same = src->dims[d] == dst->dims[d];
    if (!same) return fail(HPVM_ERR_INVALID_GRAPH, "a one-to-one edge needs identical grids");
  }
  auto e = std::make_unique<hpvm_edge>(hpvm_edge{src, dst, repl, sp, dp, stream != 0});
  hpvm_edge* raw = e.get();
  src->ctx->edges.push_back(std::move(e));
  src->parent->edges.push_back(raw);
  src->ctx->structure++;
  if (out) *out = raw;
  return ok();
}

int hpvm_bind_input(hpvm_node* child, int ip, int ic, int stream) {
  if (!child) return fail(HPVM_ERR_INVALID_ARG, "node is NULL");
  if (!child->parent) return fail(HPVM_ERR_INVALID_GRAPH, "the root has no parent to bind from");
  if (ip < 0 || ip >= in_arity(child->parent))
    return fail(HPVM_ERR_INVALID_ARG, "parent input %d is out of range", ip);
  if (ic < 0 || ic >= in_arity(child))
    return fail(HPVM_ERR_INVALID_ARG, "input %d of %s is out of range", ic, node_label(child).c_str());
  child->parent->in_binds.push_back(Bind{child, ip, ic, stream != 0});
  child->ctx->structure++;
  return ok();
}

int hpvm_bind_output(hpvm_node* child, int oc, int op, int stream) {
  if (!child) return fail(HPVM_ERR_INVALID_ARG, "node is NULL");
  if (!child->parent) return fail(HPVM_ERR_INVALID_GRAPH, "the root has no parent to bind to");
  if (oc < 0 || oc >= out_arity(child))
    return fail(HPVM_ERR_INVALID_ARG, "output %d of %s is out of range", oc, node_label(child).c_str());
  if (op < 0 || op >= out_arity(child->parent))
    return fail(HPVM_ERR_INVALID_ARG, "parent output %d is out of range", op);
  for (auto& b : child->parent->out_binds)
    if (b.outer == op) return fail(HPVM_ERR_INVALID_GRAPH, "parent output %d is already bound", op);
  child->parent->out_binds.push_back(Bind{child, op, oc, stream != 0});
  child->ctx->structure++;
  return ok();
}

int hpvm_get_parent_node(hpvm_node* node, hpvm_node** out) {
  if (!node || !out) return fail(HPVM_ERR_INVALID_ARG, "node or out is NULL");
  *out = node->parent;
  return ok();
}

int hpvm_get_num_dims(hpvm_node* node, int* out) {
  if (!node || !out) return fail(HPVM_ERR_INVALID_ARG, "node or out is NULL");
  *out = node->ndims;
  return ok();
}

int hpvm_get_num_node_instances(hpvm_node* node, int dim, int64_t* out) {
  if (!node || !out) return fail(HPVM_ERR_INVALID_ARG, "node or out is NULL");
  if (dim < 0 || dim > 2) return fail(HPVM_ERR_INVALID_ARG, "dim must be 0, 1 or 2");
  *out = dim < node->ndims ? node->dims[dim] : 1;
  return ok();
}

int hpvm_validate(hpvm_node* root) {
  if (!root) return fail(HPVM_ERR_INVALID_ARG, "root is NULL");
  if (root->parent) return fail(HPVM_ERR_INVALID_GRAPH, "not a root node");
  if (root->kind != HPVM_NODE_INTERNAL || root->ndims != 0)
    return fail(HPVM_ERR_INVALID_GRAPH, "the root must be a single-instance internal node");
  int rc = validate_node(root);
  return rc == HPVM_OK ? ok() : rc;
}

int hpvm_plan_sgemm(int tier, int64_t M, int64_t N, int64_t K, int32_t* block_x, int32_t* block_y,
                    int32_t* grid_x, int32_t* grid_y) {
  (void)K;
  if (!block_x || !block_y || !grid_x || !grid_y) return fail(HPVM_ERR_INVALID_ARG, "NULL output");
  if (M < 0 || N < 0) return fail(HPVM_ERR_SHAPE, "negative M or N");
  int tm = 16, tn = 16;
  switch (tier) {
    case HPVM_TIER_FP32_DFG: tm = tn = 16; break;
    case HPVM_TIER_FP32: hpvm::fp32_tiled_tile(&tm, &tn); break;
    case HPVM_TIER_BF16X3:
    case HPVM_TIER_BF16:
    case HPVM_TIER_FP8:
    case HPVM_TIER_BF16X6: hpvm::tc_tile(tier, &tm, &tn); break;
    default: return fail(HPVM_ERR_INVALID_ARG, "unknown tier %d", tier);
  }
  *block_x = tm;
  *block_y = tn;
  *grid_x = (int32_t)std::max<int64_t>(1, (M + tm - 1) / tm);
  *grid_y = (int32_t)std::max<int64_t>(1, (N + tn - 1) / tn);
  return ok();
}

int hpvm_workspace_size(hpvm_ctx* ctx, hpvm_node* root, const void* args, size_t args_size, size_t* out) {
  if (!ctx || !out) return fail(HPVM_ERR_INVALID_ARG, "ctx or out is NULL");
  Plan P;
  int rc = lower_graph(root, args, args_size, &P);
  if (rc != HPVM_OK) return rc;
  *out = plan_workspace(P);
  return ok();
}

int hpvm_set_workspace(hpvm_ctx* ctx, void* dev_ptr, size_t bytes) {
  if (!ctx) return fail(HPVM_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->device < 0) return fail(HPVM_ERR_NO_DEVICE, "host-only context");
  if (dev_ptr && (reinterpret_cast<uintptr_t>(dev_ptr) & 255u))
    return fail(HPVM_ERR_ALIGN, "workspace must be 256-byte aligned");
  if (ctx->ws && ctx->ws_owned) {
    cudaDeviceSynchronize();
    cudaFree(ctx->ws);
  }
  ctx->ws = dev_ptr;
  ctx->ws_bytes = dev_ptr ? bytes : 0;
  ctx->ws_owned = false;
  return ok();
}

int hpvm_plane_cache_bytes(hpvm_ctx* ctx, int64_t* bytes) {
  if (!ctx || !bytes) return fail(HPVM_ERR_INVALID_ARG, "ctx or bytes is NULL");
  *bytes = (int64_t)ctx->plane_bytes;
  return ok();
}

int hpvm_drop_planes(hpvm_ctx* ctx) {
  if (!ctx) return fail(HPVM_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->device >= 0) {
    cudaSetDevice(ctx->device);
    free_planes(ctx);
  }
  return ok();
}

int hpvm_launch(hpvm_ctx* ctx, hpvm_node* root, const void* args, size_t args_size, int stream_graph,
                void* cuda_stream, hpvm_graph** out) {
  if (out) *out = nullptr;
  if (!ctx || !out) return fail(HPVM_ERR_INVALID_ARG, "ctx or out is NULL");
  if (root && root->ctx != ctx) return fail(HPVM_ERR_INVALID_ARG, "root belongs to another context");
  Plan P;
  int rc = lower_graph(root, args, args_size, &P);
  if (rc != HPVM_OK) return rc;
  for (auto& S : P.stages)
    if ((rc = check_stage_tier(S, record_i32(P, S.rec, kTierOffset))) != HPVM_OK) return rc;
  if (ctx->device < 0) return fail(HPVM_ERR_NO_DEVICE, "host-only context cannot launch");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  auto g = std::make_unique<hpvm_graph>();
  g->ctx = ctx;
  g->stream = s;
  g->root = root;
  if (stream_graph) {
    g->validated = ctx->structure;  // lower_graph above validated the structure
    // A streaming graph stays alive: nothing runs now; every hpvm_push runs
    // one item on the next stream of the ring, after the work enqueued on
    // the caller's stream before this launch.
    g->streaming = true;
    cudaEvent_t start;
    if ((e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
    cudaEventRecord(start, s);
    g->slots.assign(kStreamSlots, nullptr);
    g->slot_ws.assign(kStreamSlots, nullptr);
    g->slot_ws_bytes.assign(kStreamSlots, 0);
    for (int i = 0; i < kStreamSlots; ++i) {
      if (!ctx->spare_streams.empty()) {
        g->slots[i] = ctx->spare_streams.back();
        ctx->spare_streams.pop_back();
      } else if ((e = cudaStreamCreateWithFlags(&g->slots[i], cudaStreamNonBlocking)) != cudaSuccess) {
        cudaEventDestroy(start);
        free_graph(g.release());
        return cuda_fail(e, "cudaStreamCreate");
      }
      cudaStreamWaitEvent(g->slots[i], start, 0);
      if (!ctx->spare_ws.empty()) {
        g->slot_ws[i] = ctx->spare_ws.back().first;
        g->slot_ws_bytes[i] = ctx->spare_ws.back().second;
        ctx->spare_ws.pop_back();
      }
    }
    cudaEventDestroy(start);
    *out = g.get();
    ctx->graphs.insert(g.release());
    return ok();
  }
  void* ws = nullptr;
  size_t ws_bytes = 0;
  const size_t ws_need = plan_workspace(P);
  if ((rc = ensure_workspace(ctx, ws_need, &ws, &ws_bytes)) != HPVM_OK) return rc;
  // Launches of one context share its workspace. A launch on a stream other
  // than the previous workspace user's first waits for that launch, so the
  // two never overlap on the GPU. Inside stream capture the caller orders
  // captured launches (an event recorded outside a capture cannot be waited
  // on inside it), so nothing is added there.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const bool order_ws = ws_need > 0 && cudaStreamIsCapturing(s, &cap) == cudaSuccess &&
                        cap == cudaStreamCaptureStatusNone;
  if (order_ws && ctx->ws_event && ctx->ws_stream != s) {
    if ((e = cudaStreamWaitEvent(s, ctx->ws_event, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
  }
  if ((rc = execute_plan(ctx, P, s, ws, ws_bytes, &g->info)) != HPVM_OK) return rc;
  if (order_ws) {
    if (!ctx->ws_event && (e = cudaEventCreateWithFlags(&ctx->ws_event, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
    if ((e = cudaEventRecord(ctx->ws_event, s)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    ctx->ws_stream = s;
  }
  const int flags = record_i32(P, P.stages.front().rec, kFlagsOffset);
  if (!(flags & HPVM_LAUNCH_NO_EVENT)) {
    e = cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    e = cudaEventRecord(g->done, s);
    if (e != cudaSuccess) {
      cudaEventDestroy(g->done);
      g->done = nullptr;
      return cuda_fail(e, "cudaEventRecord");
    }
  }
  *out = g.get();
  ctx->graphs.insert(g.release());
  return ok();
}

int hpvm_push(hpvm_graph* g, const void* args, size_t args_size) {
  if (!g || !args) return fail(HPVM_ERR_INVALID_ARG, "graph or args is NULL");
  hpvm_ctx* ctx = g->ctx;
  if (!ctx->graphs.count(g)) return fail(HPVM_ERR_INVALID_ARG, "unknown or finished graph handle");
  if (!g->streaming) return fail(HPVM_ERR_INVALID_ARG, "push needs a graph launched as a streaming graph");
  int rc;
  if (g->coalesce <= 1 || g->validated != ctx->structure) {
    // the structure is validated again when it changed since the last check;
    // a coalescing graph lowers its records when their group is launched
    Plan P;
    if ((rc = lower_graph(g->root, args, args_size, &P, g->validated == ctx->structure)) != HPVM_OK) return rc;
    g->validated = ctx->structure;
  } else if (!args || args_size < kRecBytes) {
    return fail(HPVM_ERR_INVALID_ARG, "argument record too small (%zu < %zu bytes)", args_size, kRecBytes);
  }
  cudaSetDevice(ctx->device);
  StreamItem it;
  it.record.assign(static_cast<const uint8_t*>(args), static_cast<const uint8_t*>(args) + args_size);
  g->items.push_back(std::move(it));
  g->pushed++;
  if (g->coalesce <= 1) {
    if ((rc = launch_item(g, g->items.back())) != HPVM_OK) {
      g->items.pop_back();
      return rc;
    }
    return ok();
  }
  size_t waiting = 0;
  for (auto& q : g->items) waiting += !q.launched;
  if ((int)waiting >= g->coalesce && (rc = flush_items(g)) != HPVM_OK) return rc;
  return ok();
}

int hpvm_pop(hpvm_graph* g, void* out, size_t out_size, int64_t timeout_ms) {
  if (!g) return fail(HPVM_ERR_INVALID_ARG, "graph is NULL");
  hpvm_ctx* ctx = g->ctx;
  if (!ctx->graphs.count(g)) return fail(HPVM_ERR_INVALID_ARG, "unknown or finished graph handle");
  if (!g->streaming) return fail(HPVM_ERR_INVALID_ARG, "pop needs a graph launched as a streaming graph");
  if (g->items.empty()) return fail(HPVM_ERR_INVALID_ARG, "pop on a stream with no pushed item");
  cudaSetDevice(ctx->device);
  if (!g->items.front().launched) {
    int rc0 = flush_items(g);
    if (rc0 != HPVM_OK) return rc0;
  }
  StreamItem& it = g->items.front();
  int rc = wait_event(it.done, timeout_ms);
  if (rc == HPVM_ERR_TIMEOUT) return rc;  // the item stays queued
  if (rc == HPVM_OK) rc = check_status(ctx);
  if (out && out_size) memcpy(out, it.record.data(), std::min(out_size, it.record.size()));
  if (rc == HPVM_OK) g->spare_events.push_back(it.done);  // completed: reusable
  else cudaEventDestroy(it.done);
  g->items.pop_front();
  return rc == HPVM_OK ? ok() : rc;
}

int hpvm_wait(hpvm_graph* g, int64_t timeout_ms) {
  if (!g) return fail(HPVM_ERR_INVALID_ARG, "graph is NULL");
  hpvm_ctx* ctx = g->ctx;
  if (!ctx->graphs.count(g)) return fail(HPVM_ERR_INVALID_ARG, "unknown or already finished graph handle");
  cudaSetDevice(ctx->device);
  int rc = HPVM_OK;
  if (g->streaming) {
    // items still queued run now; if that fails, the launched ones are
    // still waited for before the graph is freed
    const int frc = flush_items(g);
    for (auto& it : g->items) {
      if (!it.launched) continue;
      rc = wait_event(it.done, timeout_ms);
      if (rc == HPVM_ERR_TIMEOUT) return rc;
      if (rc != HPVM_OK) break;
    }
    if (rc == HPVM_OK && frc != HPVM_OK) rc = frc;
  } else if (g->done) {
    rc = wait_event(g->done, timeout_ms);
    if (rc == HPVM_ERR_TIMEOUT) return rc;
  } else {
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "waiting for the graph");
  }
  if (rc == HPVM_OK) rc = check_status(ctx);
  ctx->graphs.erase(g);
  free_graph(g, g->streaming && rc == HPVM_OK);  // a finished streaming graph's streams serve the next one
  return rc == HPVM_OK ? ok() : rc;
}

int hpvm_set_wait_limit(hpvm_ctx* ctx, int64_t limit_us) {
  if (!ctx) return fail(HPVM_ERR_INVALID_ARG, "ctx is NULL");
  if (limit_us < 0 || limit_us > 10000000)
    return fail(HPVM_ERR_INVALID_ARG, "wait limit %lld us is outside 0..10^7", (long long)limit_us);
  ctx->status.wait_limit_us = (uint32_t)limit_us;
  return ok();
}

int hpvm_stream_coalesce(hpvm_graph* g, int items) {
  if (!g || items < 1) return fail(HPVM_ERR_INVALID_ARG, "graph is NULL or items < 1");
  if (!g->ctx->graphs.count(g)) return fail(HPVM_ERR_INVALID_ARG, "unknown or finished graph handle");
  if (!g->streaming) return fail(HPVM_ERR_INVALID_ARG, "coalescing applies to a streaming graph");
  g->coalesce = items;
  if (items == 1) {
    cudaSetDevice(g->ctx->device);
    return flush_items(g) == HPVM_OK ? ok() : HPVM_ERR_CUDA;
  }
  return ok();
}

int hpvm_graph_info(hpvm_graph* g, hpvm_launch_info* out) {
  if (!g || !out) return fail(HPVM_ERR_INVALID_ARG, "graph or out is NULL");
  if (!g->ctx->graphs.count(g)) return fail(HPVM_ERR_INVALID_ARG, "unknown or finished graph handle");
  *out = g->info;
  return ok();
}

int hpvm_set_kernel_timing(hpvm_ctx* ctx, int enable) {
  if (!ctx) return fail(HPVM_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->device < 0) return fail(HPVM_ERR_NO_DEVICE, "host-only context");
  ctx->timing = enable != 0;
  return ok();
}

int hpvm_kernel_timing(hpvm_ctx* ctx, double* total_ms, int64_t* launches) {
  if (!ctx || !total_ms || !launches) return fail(HPVM_ERR_INVALID_ARG, "NULL argument");
  double sum = 0.0;
  int64_t n = 0;
  int rc = HPVM_OK;
  for (auto& pr : ctx->timed) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(pr.second);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
    if (e != cudaSuccess && rc == HPVM_OK) rc = cuda_fail(e, "reading kernel timing events");
    sum += ms;
    ++n;
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  ctx->timed.clear();
  *total_ms = sum;
  *launches = n;
  return rc == HPVM_OK ? ok() : rc;
}

int hpvm_track_mem(hpvm_ctx* ctx, void* p, int64_t bytes) {
  if (!ctx || !p) return fail(HPVM_ERR_INVALID_ARG, "ctx or pointer is NULL");
  if (bytes <= 0) return fail(HPVM_ERR_INVALID_ARG, "size must be positive");
  char* c = static_cast<char*>(p);
  for (auto& t : ctx->tracked) {
    if (t.host == c) {
      if (t.bytes != bytes) {
        if (t.dev) {
          cudaDeviceSynchronize();
          cudaFree(t.dev);
        }
        t.dev = nullptr;
        t.bytes = bytes;
      }
      t.host_valid = true;
      t.dev_valid = false;  // the host copy is now the latest
      return ok();
    }
    if (c < t.host + t.bytes && t.host < c + bytes)
      return fail(HPVM_ERR_INVALID_ARG, "region overlaps a tracked region");
  }
  TrackEntry t;
  t.host = c;
  t.bytes = bytes;
  ctx->tracked.push_back(t);
  return ok();
}

int hpvm_request_mem(hpvm_ctx* ctx, void* p, int64_t bytes) {
  if (!ctx || !p) return fail(HPVM_ERR_INVALID_ARG, "ctx or pointer is NULL");
  int64_t off = 0;
  TrackEntry* t = find_tracked(ctx, p, &off);
  if (!t) return fail(HPVM_ERR_INVALID_ARG, "pointer is not in a tracked region");
  if (bytes < 0 || off + bytes > t->bytes) return fail(HPVM_ERR_SHAPE, "request beyond the tracked region");
  if (t->host_valid) return ok();
  if (ctx->device < 0) return fail(HPVM_ERR_NO_DEVICE, "host-only context");
  cudaSetDevice(ctx->device);
  // wait for the launch that last wrote the region (other streams and
  // contexts keep running), then copy on the context's own stream
  cudaError_t e = t->written_set ? cudaEventSynchronize(t->written) : cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "waiting before device->host copy");
  if (!ctx->copy_stream && (e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "creating the copy stream");
  e = cudaMemcpyAsync(t->host, t->dev, (size_t)t->bytes, cudaMemcpyDeviceToHost, ctx->copy_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->copy_stream);
  if (e != cudaSuccess) return cuda_fail(e, "device->host copy");
  t->host_valid = true;
  return ok();
}

int hpvm_untrack_mem(hpvm_ctx* ctx, void* p) {
  if (!ctx || !p) return fail(HPVM_ERR_INVALID_ARG, "ctx or pointer is NULL");
  for (size_t i = 0; i < ctx->tracked.size(); ++i) {
    if (ctx->tracked[i].host == p) {
      if (ctx->tracked[i].dev) {
        cudaSetDevice(ctx->device);
        cudaDeviceSynchronize();
        cudaFree(ctx->tracked[i].dev);
      }
      if (ctx->tracked[i].written) cudaEventDestroy(ctx->tracked[i].written);
      ctx->tracked.erase(ctx->tracked.begin() + (long)i);
      return ok();
    }
  }
  return fail(HPVM_ERR_INVALID_ARG, "pointer is not the start of a tracked region");
}

int hpvm_selftest_wait_timeout(hpvm_ctx* ctx, int64_t limit_ms, void* cuda_stream) {
  if (!ctx) return fail(HPVM_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->device < 0) return fail(HPVM_ERR_NO_DEVICE, "host-only context");
  if (limit_ms < 1 || limit_ms > 10000) return fail(HPVM_ERR_INVALID_ARG, "limit must be 1..10000 ms");
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = hpvm::launch_wait_selftest(ctx->status, (uint64_t)limit_ms * 1000000ull, s);
  if (e != cudaSuccess) return cuda_fail(e, "self-test launch");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "self-test wait");
  int rc = check_status(ctx);
  return rc == HPVM_OK ? ok() : rc;
}

// ---- batches -----------------------------------------------------------------
namespace {
uint64_t batch_signature(const std::vector<hpvm::SgemmDesc>& d, int tier) {
  uint64_t h = 1469598103934665603ull ^ (uint64_t)tier;
  auto mix = [&](uint64_t v) {
    h ^= v;
    h *= 1099511628211ull;
  };
  for (auto& x : d) {
    mix((uint64_t)x.M);
    mix((uint64_t)x.N);
    mix((uint64_t)x.K);
    mix((uint64_t)(x.transA * 2 + x.transB));
  }
  return h;
}
}  // namespace

int hpvm_batch_plan(int count, const int64_t* M, const int64_t* N, const int64_t* K, int policy, int32_t* bn,
                    int32_t* tiles, int64_t tile_cap, int64_t* num_tiles) {
  if (count < 0 || (count > 0 && (!M || !N || !K)) || !num_tiles)
    return fail(HPVM_ERR_INVALID_ARG, "bad arguments");
  if (policy < 0 || policy > 11) return fail(HPVM_ERR_INVALID_ARG, "policy must be 0..11");
  std::vector<hpvm::SgemmDesc> d(count);
  for (int i = 0; i < count; ++i) {
    if (M[i] < 0 || N[i] < 0 || K[i] < 0) return fail(HPVM_ERR_SHAPE, "negative extent in instance %d", i);
    d[i].M = M[i];
    d[i].N = N[i];
    d[i].K = K[i];
  }
  auto w = hpvm::batch_choose_bn(d, policy);
  std::vector<int> t;
  const int tm = hpvm::batch_tile_m(policy);
  hpvm::batch_schedule(d, w, tm > 128 ? std::max(1, hpvm::tc_num_sms() / 2) : hpvm::tc_num_sms(), &t, tm);
  if (bn)
    for (int i = 0; i < count; ++i) bn[i] = w[i];
  *num_tiles = (int64_t)(t.size() / 4);
  if (tiles) {
    if (tile_cap < *num_tiles) return fail(HPVM_ERR_SHAPE, "tile buffer holds %lld tiles, %lld needed",
                                           (long long)tile_cap, (long long)*num_tiles);
    for (size_t i = 0; i < t.size(); ++i) tiles[i] = t[i];
  }
  return ok();
}

int hpvm_batch_prepare(hpvm_ctx* ctx, hpvm_node* root, const void* records, size_t record_bytes, int count,
                       int policy, hpvm_batch** out) {
  if (out) *out = nullptr;
  if (!ctx || !out || !records || count <= 0) return fail(HPVM_ERR_INVALID_ARG, "bad arguments");
  if (policy < -1 || policy > 11) return fail(HPVM_ERR_INVALID_ARG, "policy must be -1 (tuned) or 0..11");
  if (ctx->device < 0) return fail(HPVM_ERR_NO_DEVICE, "host-only context");
  cudaSetDevice(ctx->device);
  std::vector<hpvm::SgemmDesc> d(count);
  int tier = -1, rc;
  for (int i = 0; i < count; ++i) {
    Plan P;
    const uint8_t* rec = static_cast<const uint8_t*>(records) + (size_t)i * record_bytes;
    if ((rc = lower_graph(root, rec, record_bytes, &P)) != HPVM_OK) return rc;
    if (P.stages.size() != 1 || P.stages[0].epi.kind)
      return fail(HPVM_ERR_UNSUPPORTED, "a batch runs single-stage sgemm graphs without elementwise leaves");
    const int t = record_i32(P, P.stages[0].rec, kTierOffset);
    if (t != HPVM_TIER_BF16X3 && t != HPVM_TIER_BF16)
      return fail(HPVM_ERR_UNSUPPORTED, "a batch runs the BF16X3 or BF16 tier (instance %d has tier %d)", i, t);
    if (tier >= 0 && t != tier) return fail(HPVM_ERR_UNSUPPORTED, "all instances of a batch need the same tier");
    tier = t;
    d[i] = P.stages[0].d;
    if (d[i].M > 0 && d[i].N > 0) {
      if ((rc = check_device_pointer(d[i].C, "C")) != HPVM_OK) return rc;
      if (d[i].K > 0 && ((rc = check_device_pointer(d[i].A, "A")) != HPVM_OK ||
                         (rc = check_device_pointer(d[i].B, "B")) != HPVM_OK))
        return rc;
    }
    if (d[i].M > INT32_MAX / 2 || d[i].N > INT32_MAX / 2 || d[i].K > INT32_MAX / 2)
      return fail(HPVM_ERR_SHAPE, "instance %d is too large for a batch", i);
  }
  if (policy >= 8 && tier != HPVM_TIER_BF16X3)
    return fail(HPVM_ERR_INVALID_ARG, "policies 8..11 (in-leaf conversion) take the BF16X3 tier");
  auto b = std::make_unique<hpvm_batch>();
  b->ctx = ctx;
  b->tb.tier = tier;
  b->tb.d = d;
  b->signature = batch_signature(d, tier);
  int pol = policy;
  if (pol < 0) {
    pol = 2;
    for (auto& kv : ctx->tuned)
      if (kv.first == b->signature) pol = kv.second;
  }
  b->tb.policy = pol;
  std::string err;
  if (hpvm::tc_batch_build(&b->tb, &err)) {
    hpvm::tc_batch_free(&b->tb);
    return fail(HPVM_ERR_CUDA, "batch preparation: %s", err.c_str());
  }
  *out = b.get();
  ctx->batches.insert(b.release());
  return ok();
}

int hpvm_batch_run(hpvm_batch* b, void* cuda_stream) {
  if (!b || !b->ctx->batches.count(b)) return fail(HPVM_ERR_INVALID_ARG, "unknown batch");
  hpvm_ctx* ctx = b->ctx;
  hpvm::LaunchHooks hooks;
  if (ctx->timing) {
    if (cudaEventCreate(&hooks.main_begin) != cudaSuccess || cudaEventCreate(&hooks.main_end) != cudaSuccess)
      return fail(HPVM_ERR_CUDA, "cannot create timing events");
    ctx->timed.emplace_back(hooks.main_begin, hooks.main_end);
  }
  cudaError_t e = hpvm::tc_batch_run(b->tb, ctx->status, static_cast<cudaStream_t>(cuda_stream), &hooks);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  return ok();
}

int hpvm_batch_autotune(hpvm_batch* b, void* cuda_stream, int reps, int* best_policy, double* best_ms) {
  if (!b || !b->ctx->batches.count(b)) return fail(HPVM_ERR_INVALID_ARG, "unknown batch");
  int best = -1;
  double ms = 0;
  std::string err;
  if (hpvm::tc_batch_autotune(&b->tb, b->ctx->status, static_cast<cudaStream_t>(cuda_stream), reps < 1 ? 1 : reps,
                              &best, &ms, &err))
    return fail(HPVM_ERR_CUDA, "autotuning: %s", err.c_str());
  bool found = false;
  for (auto& kv : b->ctx->tuned)
    if (kv.first == b->signature) {
      kv.second = best;
      found = true;
    }
  if (!found) b->ctx->tuned.emplace_back(b->signature, best);
  if (best_policy) *best_policy = best;
  if (best_ms) *best_ms = ms;
  return check_status(b->ctx) == HPVM_OK ? ok() : HPVM_ERR_DEVICE_FAULT;
}

int hpvm_batch_info(hpvm_batch* b, hpvm_batch_stats* out) {
  if (!b || !out || !b->ctx->batches.count(b)) return fail(HPVM_ERR_INVALID_ARG, "unknown batch or NULL out");
  memset(out, 0, sizeof *out);
  out->count = (int32_t)b->tb.d.size();
  out->tier = b->tb.tier;
  out->policy = b->tb.policy;
  out->tiles = b->tb.real_tiles;
  out->split_tiles = b->tb.convert ? b->tb.num_pre_tiles : b->tb.num_split_tiles;
  out->grid = b->tb.grid;
  out->tile_m = b->tb.tile_m;
  out->workspace_bytes = (int64_t)b->tb.ws_bytes;
  for (int w : b->tb.bn) out->tile_width_count[w == 64 ? 0 : w == 128 ? 1 : 2]++;
  return ok();
}

int hpvm_batch_free(hpvm_batch* b) {
  if (!b || !b->ctx->batches.count(b)) return fail(HPVM_ERR_INVALID_ARG, "unknown batch");
  cudaSetDevice(b->ctx->device);
  cudaDeviceSynchronize();
  hpvm::tc_batch_free(&b->tb);
  b->ctx->batches.erase(b);
  delete b;
  return ok();
}

}  // extern "C"
