// Host runtime of the C-ABI (include/hpvm.h): graph builder (the paper's
// Graph Builder pass, Section 4.2, fed by intrinsic calls instead of IR),
// validator (rules of Sections 3.1-3.2), lowering of the sgemm graph shape
// (Section 4.4 tiling, the host code of Section 5.3: Allocation size known
// before the launch, local/global work sizes from the two grids), launch and
// bounded wait, and the memory tracker of Section 3.3.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
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

constexpr int kMaxPorts = 64;

// Types of the sgemm root record fields (port p = field p).
enum FieldType { F_PTR, F_I64, F_I32, F_F32 };
constexpr int kRootPorts = 20;
constexpr FieldType kRootType[kRootPorts] = {
    F_PTR, F_I64, F_I32,  // A, bytesA, lda
    F_PTR, F_I64, F_I32,  // B, bytesB, ldb
    F_PTR, F_I64, F_I32,  // C, bytesC, ldc
    F_I32, F_F32, F_F32,  // k, alpha, beta
    F_I32, F_I32, F_I32, F_I32,  // block_x, block_y, grid_x, grid_y
    F_I32, F_I32, F_I32, F_I32,  // M, N, transA, transB
};
constexpr size_t kRootOffset[kRootPorts] = {0, 8, 16, 20, 28, 36, 40, 48, 56, 60, 64, 68,
                                            72, 76, 80, 84, 88, 92, 96, 100};
const char* kRootName[kRootPorts] = {"A", "bytesA", "lda", "B", "bytesB", "ldb", "C",
                                     "bytesC", "ldc", "k", "alpha", "beta", "block_x",
                                     "block_y", "grid_x", "grid_y", "M", "N", "transA", "transB"};

// Input ports of the SgemmLeaf node function and their types.
constexpr int kLeafPorts = 20;
constexpr FieldType kLeafType[kLeafPorts] = {
    F_PTR, F_I64, F_I32, F_PTR, F_I64, F_I32, F_PTR, F_I64, F_I32,  // A..ldc
    F_I32, F_F32, F_F32,                                            // k, alpha, beta
    F_PTR, F_I64, F_PTR, F_I64,  // shB, bytesShB, shA, bytesShA (Allocation)
    F_I32, F_I32, F_I32, F_I32,  // M, N, transA, transB
};
// Leaf port -> the root field with the same meaning (for the data ports)
constexpr int kLeafMeaning[kLeafPorts] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11,
                                          -1, -1, -1, -1, 16, 17, 18, 19};
constexpr int kAllocInPorts = 2, kAllocOutPorts = 4;
constexpr FieldType kAllocOutType[kAllocOutPorts] = {F_PTR, F_I64, F_PTR, F_I64};

const char* kind_name(int k) {
  switch (k) {
    case HPVM_NODE_INTERNAL: return "internal";
    case HPVM_NODE_ALLOCATION: return "Allocation";
    case HPVM_NODE_SGEMM_LEAF: return "SgemmLeaf";
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

struct Bind {
  hpvm_node* child;
  int ip, ic, stream;
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
  std::vector<Bind> in_binds;      // parent input -> child input
  std::vector<Bind> out_binds;     // child output -> parent output
};

struct TrackEntry {
  char* host = nullptr;
  int64_t bytes = 0;
  void* dev = nullptr;
  bool host_valid = true, dev_valid = false;
};

struct hpvm_graph {
  hpvm_ctx* ctx = nullptr;
  cudaEvent_t done = nullptr;
  cudaStream_t stream = nullptr;
  hpvm_launch_info info{};
};

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
  hpvm::DeviceStatus status;
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> timed;  // main-kernel events
};

// ---------------------------------------------------------------------------
// helpers
namespace {

int in_arity(const hpvm_node* n) {
  switch (n->kind) {
    case HPVM_NODE_SGEMM_LEAF: return kLeafPorts;
    case HPVM_NODE_ALLOCATION: return kAllocInPorts;
    default: return n->parent == nullptr ? kRootPorts : kMaxPorts;
  }
}
int out_arity(const hpvm_node* n) {
  switch (n->kind) {
    case HPVM_NODE_SGEMM_LEAF: return 0;
    case HPVM_NODE_ALLOCATION: return kAllocOutPorts;
    default: return kMaxPorts;
  }
}
bool is_leaf(const hpvm_node* n) { return n->kind != HPVM_NODE_INTERNAL; }

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
    if (b.child == child && b.ic < (int)cnt.size()) cnt[b.ic]++;
  return cnt;
}

// ports of `n` that something under it reads (bindings to its children and
// replication extents of its children)
std::vector<bool> used_inputs(const hpvm_node* n) {
  std::vector<bool> used(kMaxPorts, false);
  for (auto& b : n->in_binds)
    if (b.ip >= 0 && b.ip < kMaxPorts) used[b.ip] = true;
  for (auto* c : n->children)
    for (int d = 0; d < c->ndims; ++d)
      if (c->dims[d] < 0) {
        int64_t p = -1 - c->dims[d];
        if (p < kMaxPorts) used[p] = true;
      }
  return used;
}

int validate_node(const hpvm_node* n) {
  if (is_leaf(n)) {
    if (!n->children.empty())
      return fail(HPVM_ERR_INVALID_GRAPH, "%s: a leaf node has children", node_label(n).c_str());
    return HPVM_OK;
  }
  // edges among children
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
  // no cycle of ordinary edges (DFS over children)
  {
    std::vector<int> state(n->children.size(), 0);
    auto index_of = [&](const hpvm_node* c) {
      for (size_t i = 0; i < n->children.size(); ++i)
        if (n->children[i] == c) return (int)i;
      return -1;
    };
    std::vector<std::pair<int, size_t>> stack;
    for (size_t r = 0; r < n->children.size(); ++r) {
      if (state[r]) continue;
      stack.push_back({(int)r, 0});
      state[r] = 1;
      while (!stack.empty()) {
        auto& [u, ei] = stack.back();
        if (ei >= n->edges.size()) {
          state[u] = 2;
          stack.pop_back();
          continue;
        }
        auto* e = n->edges[ei++];
        if (e->src != n->children[u]) continue;
        int v = index_of(e->dst);
        if (v < 0) continue;
        if (state[v] == 1) return fail(HPVM_ERR_INVALID_GRAPH, "cycle of edges under %s", node_label(n).c_str());
        if (state[v] == 0) {
          state[v] = 1;
          stack.push_back({v, 0});
        }
      }
    }
  }
  // every input a child reads is fed exactly once
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
        if (used[p] && cnt[p] == 0)
          return fail(HPVM_ERR_INVALID_GRAPH, "input %d of %s is read but never fed", p,
                      node_label(c).c_str());
        if (cnt[p] > 1)
          return fail(HPVM_ERR_INVALID_GRAPH, "input %d of %s is fed %d times", p, node_label(c).c_str(),
                      cnt[p]);
      }
    }
    int rc = validate_node(c);
    if (rc != HPVM_OK) return rc;
  }
  return HPVM_OK;
}

// ---- value resolution for lowering --------------------------------------
// Where the value of an input port comes from: a root record field, or an
// output of an Allocation node.
struct Source {
  int root_field = -1;
  hpvm_node* alloc = nullptr;
  int alloc_out = -1;
};

bool input_source(const hpvm_node* n, int port, Source* out);

// value of input `port` of internal node `n` (root: the record field)
bool value_of_input(const hpvm_node* n, int port, Source* out) {
  if (n->parent == nullptr) {
    if (port < 0 || port >= kRootPorts) return false;
    out->root_field = port;
    return true;
  }
  return input_source(n, port, out);
}

bool input_source(const hpvm_node* n, int port, Source* out) {
  const hpvm_node* par = n->parent;
  if (!par) return value_of_input(n, port, out);
  for (auto* e : par->edges)
    if (e->dst == n && e->dp == port) {
      if (e->src->kind != HPVM_NODE_ALLOCATION) return false;
      out->alloc = e->src;
      out->alloc_out = e->sp;
      return true;
    }
  for (auto& b : par->in_binds)
    if (b.child == n && b.ic == port) return value_of_input(par, b.ip, out);
  return false;
}

struct RootRecord {
  const uint8_t* base;
  template <class T>
  T get(int field) const {
    T v;
    memcpy(&v, base + kRootOffset[field], sizeof(T));
    return v;
  }
};

bool extent_of(const hpvm_node* n, int d, const RootRecord& rec, int64_t* out) {
  if (d >= n->ndims) {
    *out = 1;
    return true;
  }
  if (n->dims[d] > 0) {
    *out = n->dims[d];
    return true;
  }
  Source s;
  if (!value_of_input(n->parent, (int)(-1 - n->dims[d]), &s) || s.root_field < 0) return false;
  if (kRootType[s.root_field] != F_I32) return false;
  *out = rec.get<int32_t>(s.root_field);
  return true;
}

// The lowered sgemm graph.
struct Lowered {
  hpvm::SgemmDesc d;
  int64_t bytesA = 0, bytesB = 0, bytesC = 0;
  int64_t block_x = 0, block_y = 0, grid_x = 0, grid_y = 0;
  int64_t alloc_bx = 0, alloc_by = 0;
  bool has_a_tile = false;
};

int lower_sgemm(hpvm_node* root, const void* args, size_t args_size, Lowered* L) {
  if (!root || root->parent != nullptr)
    return fail(HPVM_ERR_INVALID_ARG, "launch needs the root node of a graph");
  if (root->kind != HPVM_NODE_INTERNAL || root->ndims != 0)
    return fail(HPVM_ERR_INVALID_GRAPH, "the root must be a single-instance internal node");
  if (!args || args_size < HPVM_SGEMM_ROOT_ARGS_BYTES)
    return fail(HPVM_ERR_INVALID_ARG, "argument record too small (%zu < %d bytes)", args_size,
                HPVM_SGEMM_ROOT_ARGS_BYTES);
  int rc = validate_node(root);
  if (rc != HPVM_OK) return rc;
  // root -> one internal 2-D grid -> {Allocation (1 instance), SgemmLeaf (2-D)}
  if (root->children.size() != 1 || root->children[0]->kind != HPVM_NODE_INTERNAL ||
      root->children[0]->ndims != 2)
    return fail(HPVM_ERR_UNSUPPORTED, "root must hold exactly one 2-D internal node (the tile grid)");
  hpvm_node* inner = root->children[0];
  hpvm_node* alloc = nullptr;
  hpvm_node* leaf = nullptr;
  for (auto* c : inner->children) {
    if (c->kind == HPVM_NODE_ALLOCATION && !alloc) alloc = c;
    else if (c->kind == HPVM_NODE_SGEMM_LEAF && !leaf) leaf = c;
    else return fail(HPVM_ERR_UNSUPPORTED, "the tile node must hold one Allocation and one SgemmLeaf");
  }
  if (!alloc || !leaf) return fail(HPVM_ERR_UNSUPPORTED, "the tile node must hold one Allocation and one SgemmLeaf");
  if (alloc->ndims != 0) return fail(HPVM_ERR_UNSUPPORTED, "the Allocation node must have one instance");
  if (leaf->ndims != 2) return fail(HPVM_ERR_UNSUPPORTED, "the SgemmLeaf must be a 2-D grid");
  for (auto* e : inner->edges) {
    if (e->stream) return fail(HPVM_ERR_UNSUPPORTED, "streaming edges are not lowered");
    if (!(e->src == alloc && e->dst == leaf && e->repl == HPVM_ALL_TO_ALL))
      return fail(HPVM_ERR_UNSUPPORTED, "only all-to-all Allocation -> SgemmLeaf edges are lowered");
  }
  for (auto& b : root->in_binds)
    if (b.stream) return fail(HPVM_ERR_UNSUPPORTED, "streaming bindings are not lowered");
  for (auto& b : inner->in_binds)
    if (b.stream) return fail(HPVM_ERR_UNSUPPORTED, "streaming bindings are not lowered");

  RootRecord rec{static_cast<const uint8_t*>(args)};
  // resolve the leaf's inputs
  int64_t vals_i[kLeafPorts] = {0};
  double vals_f[kLeafPorts] = {0};
  void* vals_p[kLeafPorts] = {nullptr};
  for (int p = 0; p < kLeafPorts; ++p) {
    Source s;
    if (!input_source(leaf, p, &s))
      return fail(HPVM_ERR_INVALID_GRAPH, "SgemmLeaf input %d does not resolve to a root field or an Allocation output", p);
    if (p >= 12 && p <= 15) {
      if (!s.alloc) return fail(HPVM_ERR_UNSUPPORTED, "SgemmLeaf input %d (tile memory) must come from the Allocation node", p);
      if (kAllocOutType[s.alloc_out] != kLeafType[p])
        return fail(HPVM_ERR_INVALID_GRAPH, "Allocation output %d has the wrong type for SgemmLeaf input %d", s.alloc_out, p);
      if ((p == 12 && s.alloc_out != 0) || (p == 13 && s.alloc_out != 1))
        return fail(HPVM_ERR_UNSUPPORTED, "SgemmLeaf inputs 12, 13 must be Allocation outputs 0, 1");
      if (p == 14 || p == 15) L->has_a_tile = true;
      continue;
    }
    if (s.root_field < 0)
      return fail(HPVM_ERR_UNSUPPORTED, "SgemmLeaf input %d must come from the root record", p);
    if (kRootType[s.root_field] != kLeafType[p])
      return fail(HPVM_ERR_INVALID_GRAPH, "SgemmLeaf input %d is bound to root field %s of another type", p,
                  kRootName[s.root_field]);
    switch (kLeafType[p]) {
      case F_PTR: vals_p[p] = rec.get<void*>(s.root_field); break;
      case F_I64: vals_i[p] = rec.get<int64_t>(s.root_field); break;
      case F_I32: vals_i[p] = rec.get<int32_t>(s.root_field); break;
      case F_F32: vals_f[p] = rec.get<float>(s.root_field); break;
    }
    (void)kLeafMeaning;
  }
  // the Allocation node's inputs (block_x, block_y)
  for (int p = 0; p < kAllocInPorts; ++p) {
    Source s;
    if (!input_source(alloc, p, &s) || s.root_field < 0 || kRootType[s.root_field] != F_I32)
      return fail(HPVM_ERR_INVALID_GRAPH, "Allocation input %d must be an i32 root field", p);
    (p == 0 ? L->alloc_bx : L->alloc_by) = rec.get<int32_t>(s.root_field);
  }
  if (!extent_of(leaf, 0, rec, &L->block_x) || !extent_of(leaf, 1, rec, &L->block_y) ||
      !extent_of(inner, 0, rec, &L->grid_x) || !extent_of(inner, 1, rec, &L->grid_y))
    return fail(HPVM_ERR_INVALID_GRAPH, "a replication extent does not resolve to an i32 root field");

  auto& d = L->d;
  d.A = static_cast<const float*>(vals_p[0]);
  L->bytesA = vals_i[1];
  d.lda = vals_i[2];
  d.B = static_cast<const float*>(vals_p[3]);
  L->bytesB = vals_i[4];
  d.ldb = vals_i[5];
  d.C = static_cast<float*>(vals_p[6]);
  L->bytesC = vals_i[7];
  d.ldc = vals_i[8];
  d.K = vals_i[9];
  d.alpha = (float)vals_f[10];
  d.beta = (float)vals_f[11];
  d.M = vals_i[16];
  d.N = vals_i[17];
  d.transA = vals_i[18] != 0;
  d.transB = vals_i[19] != 0;

  // shapes
  if (d.M < 0 || d.N < 0 || d.K < 0) return fail(HPVM_ERR_SHAPE, "negative M, N or K");
  if (L->block_x <= 0 || L->block_y <= 0 || L->grid_x <= 0 || L->grid_y <= 0)
    return fail(HPVM_ERR_SHAPE, "replication extents must be positive");
  if (L->grid_x * L->block_x < d.M || L->grid_y * L->block_y < d.N)
    return fail(HPVM_ERR_SHAPE, "grid x block (%lld x %lld) does not cover M x N (%lld x %lld)",
                (long long)(L->grid_x * L->block_x), (long long)(L->grid_y * L->block_y), (long long)d.M,
                (long long)d.N);
  const int64_t ar = d.transA ? d.K : d.M, ac = d.transA ? d.M : d.K;
  const int64_t br = d.transB ? d.N : d.K, bc = d.transB ? d.K : d.N;
  if (d.lda < std::max<int64_t>(1, ar)) return fail(HPVM_ERR_SHAPE, "lda (%lld) < rows of A (%lld)", (long long)d.lda, (long long)ar);
  if (d.ldb < std::max<int64_t>(1, br)) return fail(HPVM_ERR_SHAPE, "ldb (%lld) < rows of B (%lld)", (long long)d.ldb, (long long)br);
  if (d.ldc < std::max<int64_t>(1, d.M)) return fail(HPVM_ERR_SHAPE, "ldc (%lld) < M (%lld)", (long long)d.ldc, (long long)d.M);
  auto need = [](int64_t rows, int64_t cols, int64_t ld) -> int64_t {
    return (rows == 0 || cols == 0) ? 0 : 4 * (ld * (cols - 1) + rows);
  };
  const bool work = d.M > 0 && d.N > 0;
  if (work && d.K > 0) {
    if (!d.A || !d.B) return fail(HPVM_ERR_INVALID_ARG, "A or B is NULL");
    if (L->bytesA < need(ar, ac, d.lda)) return fail(HPVM_ERR_SHAPE, "bytesA (%lld) < %lld needed", (long long)L->bytesA, (long long)need(ar, ac, d.lda));
    if (L->bytesB < need(br, bc, d.ldb)) return fail(HPVM_ERR_SHAPE, "bytesB (%lld) < %lld needed", (long long)L->bytesB, (long long)need(br, bc, d.ldb));
  }
  if (work) {
    if (!d.C) return fail(HPVM_ERR_INVALID_ARG, "C is NULL");
    if (L->bytesC < need(d.M, d.N, d.ldc)) return fail(HPVM_ERR_SHAPE, "bytesC (%lld) < %lld needed", (long long)L->bytesC, (long long)need(d.M, d.N, d.ldc));
  }
  return HPVM_OK;
}

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
int map_pointer(hpvm_ctx* ctx, const void* p, bool read, cudaStream_t s, const char* name,
                void** out, TrackEntry** entry, int64_t* h2d) {
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

int ensure_workspace(hpvm_ctx* ctx, size_t need, void** ws) {
  if (need == 0) {
    *ws = ctx->ws;
    return HPVM_OK;
  }
  if (ctx->ws && ctx->ws_bytes >= need) {
    *ws = ctx->ws;
    return HPVM_OK;
  }
  if (ctx->ws && !ctx->ws_owned)
    return fail(HPVM_ERR_SHAPE, "the workspace set with hpvm_set_workspace has %zu bytes, this launch needs %zu",
                ctx->ws_bytes, need);
  if (ctx->ws) {
    cudaDeviceSynchronize();
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&ctx->ws, need);
  if (e != cudaSuccess) {
    ctx->ws = nullptr;
    return fail(HPVM_ERR_OUT_OF_MEMORY, "workspace of %zu bytes: %s", need, cudaGetErrorString(e));
  }
  ctx->ws_bytes = need;
  ctx->ws_owned = true;
  *ws = ctx->ws;
  return HPVM_OK;
}

size_t workspace_need(const Lowered& L, int tier) {
  if (tier == HPVM_TIER_BF16X3 || tier == HPVM_TIER_BF16 || tier == HPVM_TIER_FP8)
    return hpvm::tc_workspace_bytes(L.d, tier);
  return 0;
}

}  // namespace

// ===========================================================================
// C-ABI
extern "C" {

const char* hpvm_last_error(void) { return g_last_error.c_str(); }
int hpvm_version(void) { return 100; }

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
    for (auto* g : ctx->graphs) {
      if (g->done) cudaEventDestroy(g->done);
      delete g;
    }
    for (auto& t : ctx->tracked)
      if (t.dev) cudaFree(t.dev);
    if (ctx->ws && ctx->ws_owned) cudaFree(ctx->ws);
    if (ctx->status.host) cudaFreeHost(ctx->status.host);
    for (auto& pr : ctx->timed) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  }
  delete ctx;
  return ok();
}

int hpvm_create_node(hpvm_ctx* ctx, hpvm_node* parent, int kind, int ndims, const int64_t* dims,
                     hpvm_node** out) {
  if (!ctx || !out) return fail(HPVM_ERR_INVALID_ARG, "ctx or out is NULL");
  *out = nullptr;
  if (kind != HPVM_NODE_INTERNAL && kind != HPVM_NODE_ALLOCATION && kind != HPVM_NODE_SGEMM_LEAF)
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
  if (stream) return fail(HPVM_ERR_UNSUPPORTED, "streaming edges are not supported by this runtime");
  auto e = std::make_unique<hpvm_edge>(hpvm_edge{src, dst, repl, sp, dp, stream});
  hpvm_edge* raw = e.get();
  src->ctx->edges.push_back(std::move(e));
  src->parent->edges.push_back(raw);
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
  if (stream) return fail(HPVM_ERR_UNSUPPORTED, "streaming bindings are not supported by this runtime");
  child->parent->in_binds.push_back(Bind{child, ip, ic, stream});
  return ok();
}

int hpvm_bind_output(hpvm_node* child, int oc, int op, int stream) {
  if (!child) return fail(HPVM_ERR_INVALID_ARG, "node is NULL");
  if (!child->parent) return fail(HPVM_ERR_INVALID_GRAPH, "the root has no parent to bind to");
  if (oc < 0 || oc >= out_arity(child))
    return fail(HPVM_ERR_INVALID_ARG, "output %d of %s is out of range", oc, node_label(child).c_str());
  if (op < 0 || op >= out_arity(child->parent))
    return fail(HPVM_ERR_INVALID_ARG, "parent output %d is out of range", op);
  if (stream) return fail(HPVM_ERR_UNSUPPORTED, "streaming bindings are not supported by this runtime");
  child->parent->out_binds.push_back(Bind{child, oc, op, stream});
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
    case HPVM_TIER_FP8: hpvm::tc_tile(tier, &tm, &tn); break;
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
  Lowered L;
  int rc = lower_sgemm(root, args, args_size, &L);
  if (rc != HPVM_OK) return rc;
  int32_t tier;
  memcpy(&tier, static_cast<const uint8_t*>(args) + 104, 4);
  *out = workspace_need(L, tier);
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

int hpvm_launch(hpvm_ctx* ctx, hpvm_node* root, const void* args, size_t args_size, int stream_graph,
                void* cuda_stream, hpvm_graph** out) {
  if (out) *out = nullptr;
  if (!ctx || !out) return fail(HPVM_ERR_INVALID_ARG, "ctx or out is NULL");
  if (root && root->ctx != ctx) return fail(HPVM_ERR_INVALID_ARG, "root belongs to another context");
  if (stream_graph) return fail(HPVM_ERR_UNSUPPORTED, "streaming graphs are not supported by this runtime");
  Lowered L;
  int rc = lower_sgemm(root, args, args_size, &L);
  if (rc != HPVM_OK) return rc;
  int32_t tier, flags;
  memcpy(&tier, static_cast<const uint8_t*>(args) + 104, 4);
  memcpy(&flags, static_cast<const uint8_t*>(args) + 108, 4);
  if (tier < HPVM_TIER_FP32_DFG || tier > HPVM_TIER_FP8) return fail(HPVM_ERR_INVALID_ARG, "unknown tier %d", tier);
  if (tier == HPVM_TIER_FP32_DFG) {
    if (L.block_x != L.block_y)
      return fail(HPVM_ERR_UNSUPPORTED, "the FP32_DFG lowering needs a square leaf grid (got %lld x %lld)",
                  (long long)L.block_x, (long long)L.block_y);
    if (L.block_x * L.block_y > 1024)
      return fail(HPVM_ERR_UNSUPPORTED, "the FP32_DFG lowering maps leaf instances to threads: at most 1024");
    if (!L.has_a_tile)
      return fail(HPVM_ERR_UNSUPPORTED, "the FP32_DFG lowering needs the Allocation's A tile (ports 14, 15)");
    if (L.alloc_bx * L.alloc_by < L.block_x * L.block_y)
      return fail(HPVM_ERR_SHAPE, "the Allocation tile (%lld x %lld) is smaller than the leaf grid",
                  (long long)L.alloc_bx, (long long)L.alloc_by);
  }
  if (ctx->device < 0) return fail(HPVM_ERR_NO_DEVICE, "host-only context cannot launch");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  // memory tracker: A and B are read; C is read unless beta == 0 and written
  int64_t h2d = 0;
  const bool work = L.d.M > 0 && L.d.N > 0;
  const bool need_ab = work && L.d.K > 0;
  void *A = nullptr, *B = nullptr, *C = nullptr;
  TrackEntry *tA = nullptr, *tB = nullptr, *tC = nullptr;
  if (need_ab) {
    if ((rc = map_pointer(ctx, L.d.A, true, s, "A", &A, &tA, &h2d)) != HPVM_OK) return rc;
    if ((rc = map_pointer(ctx, L.d.B, true, s, "B", &B, &tB, &h2d)) != HPVM_OK) return rc;
  }
  if (work) {
    if ((rc = map_pointer(ctx, L.d.C, L.d.beta != 0.f, s, "C", &C, &tC, &h2d)) != HPVM_OK) return rc;
  }
  hpvm::SgemmDesc d = L.d;
  d.A = static_cast<const float*>(A);
  d.B = static_cast<const float*>(B);
  d.C = static_cast<float*>(C);

  hpvm::KernelReport rep;
  if (work) {
    void* ws = nullptr;
    size_t need = workspace_need(L, tier);
    if ((rc = ensure_workspace(ctx, need, &ws)) != HPVM_OK) return rc;
    std::string err;
    hpvm::LaunchHooks hooks;
    if (ctx->timing) {
      if (cudaEventCreate(&hooks.main_begin) != cudaSuccess || cudaEventCreate(&hooks.main_end) != cudaSuccess)
        return fail(HPVM_ERR_CUDA, "cannot create timing events");
      ctx->timed.emplace_back(hooks.main_begin, hooks.main_end);
    }
    switch (tier) {
      case HPVM_TIER_FP32_DFG:
        e = hpvm::launch_fp32_dfg(d, (int)L.block_x, (int)L.grid_x, (int)L.grid_y,
                                  (size_t)(L.block_x * L.block_y * 4), s, &rep, &hooks);
        break;
      case HPVM_TIER_FP32:
        e = hpvm::launch_fp32_tiled(d, s, &rep, &hooks);
        break;
      default:
        e = hpvm::launch_tc(d, tier, ws, ctx->ws_bytes, ctx->status, s, &rep, &err, &hooks);
        if (e == cudaErrorInvalidValue && !err.empty()) return fail(HPVM_ERR_SHAPE, "%s", err.c_str());
        break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  }
  if (tC) {
    tC->dev_valid = true;
    tC->host_valid = false;
  }
  auto g = std::make_unique<hpvm_graph>();
  g->ctx = ctx;
  g->stream = s;
  if (!(flags & HPVM_LAUNCH_NO_EVENT)) {
    e = cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    e = cudaEventRecord(g->done, s);
    if (e != cudaSuccess) {
      cudaEventDestroy(g->done);
      return cuda_fail(e, "cudaEventRecord");
    }
  }
  auto& inf = g->info;
  inf.tier = tier;
  inf.kernels = rep.kernels;
  inf.grid_x = rep.grid_x;
  inf.grid_y = rep.grid_y;
  inf.grid_z = rep.grid_z;
  inf.block_threads = rep.block_threads;
  inf.tile_m = rep.tile_m;
  inf.tile_n = rep.tile_n;
  inf.tile_k = rep.tile_k;
  inf.smem_bytes = rep.smem_bytes;
  inf.literal = rep.literal;
  inf.workspace_bytes = rep.workspace_bytes;
  inf.h2d_bytes = h2d;
  inf.d2h_bytes = 0;
  *out = g.get();
  ctx->graphs.insert(g.release());
  return ok();
}

int hpvm_wait(hpvm_graph* g, int64_t timeout_ms) {
  if (!g) return fail(HPVM_ERR_INVALID_ARG, "graph is NULL");
  hpvm_ctx* ctx = g->ctx;
  if (!ctx->graphs.count(g)) return fail(HPVM_ERR_INVALID_ARG, "unknown or already finished graph handle");
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaSuccess;
  if (g->done) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      e = cudaEventQuery(g->done);
      if (e != cudaErrorNotReady) break;
      if (timeout_ms >= 0 &&
          std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms))
        return fail(HPVM_ERR_TIMEOUT, "graph not finished after %lld ms", (long long)timeout_ms);
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  } else {
    e = cudaStreamSynchronize(g->stream);
  }
  int rc = HPVM_OK;
  if (e != cudaSuccess) rc = cuda_fail(e, "waiting for the graph");
  if (rc == HPVM_OK && ctx->status.host) {
    int st = *const_cast<volatile int*>(ctx->status.host);
    if (st) {
      *const_cast<volatile int*>(ctx->status.host) = 0;
      rc = fail(HPVM_ERR_DEVICE_FAULT, "a kernel gave up a bounded wait (status bits 0x%x)", st);
    }
  }
  if (g->done) cudaEventDestroy(g->done);
  ctx->graphs.erase(g);
  delete g;
  return rc == HPVM_OK ? ok() : rc;
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
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "waiting before device->host copy");
  e = cudaMemcpy(t->host, t->dev, (size_t)t->bytes, cudaMemcpyDeviceToHost);
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
      ctx->tracked.erase(ctx->tracked.begin() + (long)i);
      return ok();
    }
  }
  return fail(HPVM_ERR_INVALID_ARG, "pointer is not the start of a tracked region");
}

}  // extern "C"
