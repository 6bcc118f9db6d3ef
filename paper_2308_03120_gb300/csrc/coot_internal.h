// Internal declarations shared by the host-side translation units of
// libcoot.so (tree parsing, code generation, run-time compilation, launch).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "coot.h"

namespace coot {

// ------------------------------------------------------------ errors

// Records `msg` as the calling thread's last error and returns `s`.
coot_status fail(coot_status s, const std::string& msg);
void clear_error();

// Whether two matrices share an element (views of one parent are compared
// by their row and column ranges; anything else by byte ranges).
bool mats_overlap(const coot_mat& a, const coot_mat& b);

// ------------------------------------------------------------ trees

struct Node {
  uint8_t op;
  uint16_t a, b;
  double imm;
};

struct Tree {
  std::vector<Node> nodes;
  int n_inputs = 0;
  int compute = COOT_F32;  // COOT_F32 or COOT_F64
  uint64_t hash = 0;       // FNV-1a of the serialised bytes
};

// Parses and validates the serialised form (format in coot.h).
coot_status parse_tree(const uint8_t* buf, size_t len, Tree* out);

// Kernel kinds (the prelude's COOT_KIND).
enum Kind {
  KIND_MAP = 0,
  KIND_REDUCE = 1,
  KIND_COLSUM = 2,
  KIND_ROWSUM = 3,
  KIND_BATCHED = 4,
  KIND_COLSTATS = 5,
  KIND_ROWSTATS = 6,
  KIND_MULTI = 7,
  KIND_DIMS = 8,
  KIND_COUNT = 9
};

// Everything that selects one compiled kernel.
struct KernelSpec {
  int kind = KIND_MAP;
  int in_dtype[4] = {0, 0, 0, 0};
  int out_dtype = 0;
  bool store = false;
  unsigned heads = 0;
  int vec = 1;
  int unroll = 1;
  int block = 256;
  bool nc = true;  // inputs read through the non-coherent path
  // several trees in one pass (KIND_MULTI): the trees (n_trees of them, all
  // over the same inputs), each one's reduction heads and its output
  // storage code (-1 when it is not stored)
  int n_trees = 0;
  const Tree* trees = nullptr;
  unsigned tree_heads[4] = {0, 0, 0, 0};
  int tree_out[4] = {-1, -1, -1, -1};
  // several trees with sums along a dimension (KIND_DIMS): the storage code
  // of tree t's column sums and row sums (-1 when not formed), and the
  // launch bound's minimum of resident blocks per SM
  int tree_cs[4] = {-1, -1, -1, -1};
  int tree_rs[4] = {-1, -1, -1, -1};
  int min_blocks = 1;
  int prefetch = 0;  // KIND_DIMS: the next column's loads in flight during the current one's
};

// Full CUDA source of one kernel: the prelude, the tree function and the
// embedded device runtime.
std::string generate_source(const Tree& t, const KernelSpec& spec);

// Name of the kernel's entry point (one per kind, so profiles tell them apart).
const char* entry_name(const KernelSpec& spec);

// ------------------------------------------------------------ JIT

// A loaded kernel (cudaKernel_t) plus its static resource use.
struct Compiled {
  void* kernel = nullptr;
  int max_blocks_per_sm = 0;
  int num_regs = 0;
};

// Returns the compiled kernel for `source`, compiling it with NVRTC on a
// miss (memory cache, then the on-disk cache, then NVRTC).
coot_status get_kernel(const std::string& source, const KernelSpec& spec, const Compiled** out);

// The kernel of (tree, spec): a lookup by digest first, then get_kernel on
// the generated source.
coot_status kernel_for(const Tree& t, const KernelSpec& spec, const Compiled** out);
void drop_kernels();

// Device facts cached by coot_init.
struct Device {
  int id = -1;
  int sm_count = 0;
  int cc_major = 0, cc_minor = 0;
  int max_threads_per_sm = 0;
};
const Device& device();
bool initialised();

uint64_t fnv1a(const void* data, size_t len, uint64_t h = 1469598103934665603ull);

// Device address of a constant 1.0 on the current device (coot_aot.cu).
coot_status device_one(const double** out);
// Device address of the bounded-wait status word (coot_aot.cu).
coot_status device_status_word(unsigned** out);

// ------------------------------------------------------------ canonical form (coot_canon.cpp)

// Whether calls on this thread canonicalise their trees (default on).
bool canonical_enabled();
void set_canonical(bool on);
// The canonical form of `in` (exact rewrites, common subexpressions,
// dead nodes dropped).  slot_alias (may be null) maps every input slot to
// the slot holding the same matrix; kept_slots (may be null) receives the
// original slots the canonical tree reads, in its new slot order (all slots
// when keep_slots is set).
void canonicalize(const Tree& in, const int* slot_alias, Tree* out, std::vector<int>* kept_slots, bool keep_slots);
// The byte form of a tree (coot.h layout).
std::vector<uint8_t> serialise(const Tree& t);

// ------------------------------------------------------------ learned launch shapes (coot_policy.cpp)

// What the cost model sees of a call.
struct CallInfo {
  int kind = KIND_MAP;
  const Tree* tree = nullptr;
  int in_bytes = 4;   // widest input storage type
  int out_bytes = 0;  // stored element-wise output, 0 if none
  unsigned heads = 0;
  int64_t n_rows = 0, n_cols = 0;
  bool dense = true;
};

// Candidate shapes {block, vec, unroll, split} of a kind; returns the count.
int candidates(int kind, const int (**out)[4]);
void call_features(const CallInfo& c, int block, int vec, int unroll, int64_t split, float* f);
bool model_ready();
int policy();
double model_predict(const float* features);

}  // namespace coot

// Launch-parameter block; identical layout to `coot_params` in jit_rt.cuh
// (every field is 8 bytes).
struct coot_params_host {
  const void* in[4];
  int64_t ld_in[4];
  void* out;
  int64_t ld_out;
  int64_t n_rows;
  int64_t n_cols;
  int64_t split;
  int64_t rows_per_split;
  unsigned char* ws;
  double* res;
  const void* plan;
  int64_t n_work;
};
static_assert(sizeof(coot_params_host) == 8 * 18, "coot_params layout");

// Launch parameters of the statistics kernels; identical layout to
// `coot_stats_params` in jit_stats.cuh.
struct coot_stats_params_host {
  coot_params_host b;
  void* out[6];
  int64_t inc[6];
  int64_t norm_type;
};
static_assert(sizeof(coot_stats_params_host) == 8 * 31, "coot_stats_params layout");

// Launch parameters of the several-tree kernel (coot_multi_params in
// jit_multi.cuh).
struct coot_multi_params_host {
  coot_params_host b;
  void* out[4];
  int64_t ld_out[4];
};

// Launch parameters of the kernel with sums along a dimension
// (coot_dims_params in jit_dims.cuh).
struct coot_dims_params_host {
  coot_params_host b;
  void* out[4];
  int64_t ld_out[4];
  void* cs[4];
  int64_t ld_cs[4];
  void* rs[4];
  int64_t n_seg;
  int64_t n_chunk;
  int64_t chunk_cols;
  int64_t cpart;
  int64_t rpart;
};
static_assert(sizeof(coot_dims_params_host) == 8 * (18 + 25), "coot_dims_params layout");

// Workspace layout (offsets in bytes), mirrored in jit_rt.cuh.
#define COOT_WS_COUNTER_OFF 128
#define COOT_WS_COUNTERS_OFF 256
#define COOT_WS_PARTIALS_OFF 65536
#define COOT_WS_MAX_COUNTERS ((COOT_WS_PARTIALS_OFF - COOT_WS_COUNTERS_OFF) / 4)
#define COOT_MAX_GRID 4096
// Elements of a batched work unit (the TMA-staged kernel's COOT_UNIT).
#define COOT_BATCH_UNIT 2048
#define COOT_MAX_ROW_CHUNKS 64
