// Serialised expression trees: parsing, validation, hashing, and the
// generation of one CUDA kernel per tree.
//
// A tree is the run-time form of Bandicoot's expression types (eOp for
// unary and scalar nodes, eGlue for binary element-wise nodes; Section 7 of
// arXiv 2308.03120).  Bandicoot evaluates such a tree node by node, each
// node's apply() launching at least one kernel (Section 7); here the whole
// tree becomes one straight-line device function that the kernels of
// jit_rt.cuh call once per element.
#include <algorithm>
#include <cinttypes>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "coot_internal.h"

extern "C" const char* coot_jit_rt_source;  // jit_rt.cuh, embedded at build time

namespace coot {

uint64_t fnv1a(const void* data, size_t len, uint64_t h) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < len; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

static uint16_t rd16(const uint8_t* p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static uint32_t rd32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static double rdf64(const uint8_t* p) {
  uint64_t u = 0;
  for (int i = 7; i >= 0; --i) u = (u << 8) | p[i];
  double d;
  std::memcpy(&d, &u, 8);
  return d;
}

static bool is_unary(int op) {
  return (op >= COOT_OP_NEG && op <= COOT_OP_SQUARE) || (op >= COOT_OP_LOG10 && op <= COOT_OP_ATAN);
}
static bool is_binary(int op) { return op >= COOT_OP_ADD && op <= COOT_OP_POW; }

coot_status parse_tree(const uint8_t* buf, size_t len, Tree* out) {
  if (buf == nullptr) return fail(COOT_ERR_INVALID_ARG, "tree is NULL");
  if (len < 16) return fail(COOT_ERR_BAD_TREE, "tree shorter than its 16-byte header");
  if (std::memcmp(buf, "COOT", 4) != 0) return fail(COOT_ERR_BAD_TREE, "tree magic is not COOT");
  const uint16_t version = rd16(buf + 4);
  const uint16_t n_nodes = rd16(buf + 6);
  const uint8_t n_inputs = buf[8];
  const uint8_t compute = buf[9];
  if (version != 1) return fail(COOT_ERR_BAD_TREE, "unknown tree version " + std::to_string(version));
  if (n_nodes < 1 || n_nodes > COOT_TREE_MAX_NODES)
    return fail(COOT_ERR_BAD_TREE, "node count " + std::to_string(n_nodes) + " outside 1..64");
  if (n_inputs < 1 || n_inputs > COOT_TREE_MAX_INPUTS)
    return fail(COOT_ERR_BAD_TREE, "input count " + std::to_string(n_inputs) + " outside 1..4");
  if (compute != COOT_F32 && compute != COOT_F64)
    return fail(COOT_ERR_BAD_TREE, "compute type must be FP32 (0) or FP64 (3)");
  if (rd16(buf + 10) != 0 || rd32(buf + 12) != 0)
    return fail(COOT_ERR_BAD_TREE, "reserved header bytes are not zero");
  if (len != 16u + 16u * n_nodes)
    return fail(COOT_ERR_BAD_TREE, "tree length does not match its node count");
  Tree t;
  t.n_inputs = n_inputs;
  t.compute = compute;
  t.nodes.resize(n_nodes);
  for (int k = 0; k < n_nodes; ++k) {
    const uint8_t* p = buf + 16 + 16 * k;
    Node nd;
    nd.op = p[0];
    nd.a = rd16(p + 2);
    nd.b = rd16(p + 4);
    nd.imm = rdf64(p + 8);
    const std::string at = "node " + std::to_string(k) + ": ";
    if (p[1] != 0 || rd16(p + 6) != 0) return fail(COOT_ERR_BAD_TREE, at + "reserved bytes are not zero");
    if (nd.op == COOT_OP_INPUT) {
      if (nd.a >= n_inputs || nd.b != 0) return fail(COOT_ERR_BAD_TREE, at + "input slot out of range");
    } else if (nd.op == COOT_OP_CONST) {
      if (nd.a != 0 || nd.b != 0) return fail(COOT_ERR_BAD_TREE, at + "constant with operands");
    } else if (is_unary(nd.op)) {
      if (nd.a >= k || nd.b != 0) return fail(COOT_ERR_BAD_TREE, at + "operand must name an earlier node");
    } else if (is_binary(nd.op)) {
      if (nd.a >= k || nd.b >= k) return fail(COOT_ERR_BAD_TREE, at + "operands must name earlier nodes");
    } else {
      return fail(COOT_ERR_BAD_TREE, at + "unknown op " + std::to_string(nd.op));
    }
    t.nodes[k] = nd;
  }
  t.hash = fnv1a(buf, len);
  *out = std::move(t);
  return COOT_OK;
}

// An exact literal of a compute-type constant: the bits of the value after
// rounding to the compute type.
static std::string literal(double v, int compute) {
  char b[64];
  if (compute == COOT_F32) {
    float f = (float)v;  // nearest FP32
    uint32_t u;
    std::memcpy(&u, &f, 4);
    std::snprintf(b, sizeof b, "__int_as_float(0x%08" PRIx32 ")", u);
  } else {
    uint64_t u;
    std::memcpy(&u, &v, 8);
    std::snprintf(b, sizeof b, "__longlong_as_double(0x%016" PRIx64 "ll)", u);
  }
  return b;
}

static std::string tree_function(const Tree& t, const char* name = "coot_f") {
  const bool f32 = t.compute == COOT_F32;
  const char* fexp = f32 ? "expf" : "exp";
  const char* flog = f32 ? "logf" : "log";
  const char* fsqrt = f32 ? "sqrtf" : "sqrt";
  const char* fabs_ = f32 ? "fabsf" : "fabs";
  std::string s = std::string("__device__ __forceinline__ COOT_REAL ") + name + "(const COOT_REAL* x) {\n";
  for (size_t k = 0; k < t.nodes.size(); ++k) {
    const Node& n = t.nodes[k];
    const std::string a = "t" + std::to_string(n.a), b = "t" + std::to_string(n.b);
    std::string e;
    switch (n.op) {
      case COOT_OP_INPUT: e = "x[" + std::to_string(n.a) + "]"; break;
      case COOT_OP_CONST: e = "(COOT_REAL)" + literal(n.imm, t.compute); break;
      case COOT_OP_NEG: e = "-" + a; break;
      case COOT_OP_ABS: e = std::string(fabs_) + "(" + a + ")"; break;
      case COOT_OP_EXP: e = std::string(fexp) + "(" + a + ")"; break;
      case COOT_OP_LOG: e = std::string(flog) + "(" + a + ")"; break;
      case COOT_OP_SQRT: e = std::string(fsqrt) + "(" + a + ")"; break;
      case COOT_OP_SQUARE: e = a + " * " + a; break;
      case COOT_OP_ADD: e = a + " + " + b; break;
      case COOT_OP_SUB: e = a + " - " + b; break;
      case COOT_OP_MUL: e = a + " * " + b; break;
      case COOT_OP_DIV: e = a + " / " + b; break;
      // relational nodes: 1 or 0 (IEEE comparisons: NaN is unordered)
      case COOT_OP_LT: e = "(" + a + " < " + b + ") ? (COOT_REAL)1 : (COOT_REAL)0"; break;
      case COOT_OP_LE: e = "(" + a + " <= " + b + ") ? (COOT_REAL)1 : (COOT_REAL)0"; break;
      case COOT_OP_GT: e = "(" + a + " > " + b + ") ? (COOT_REAL)1 : (COOT_REAL)0"; break;
      case COOT_OP_GE: e = "(" + a + " >= " + b + ") ? (COOT_REAL)1 : (COOT_REAL)0"; break;
      case COOT_OP_EQ: e = "(" + a + " == " + b + ") ? (COOT_REAL)1 : (COOT_REAL)0"; break;
      case COOT_OP_NE: e = "(" + a + " != " + b + ") ? (COOT_REAL)1 : (COOT_REAL)0"; break;
      case COOT_OP_POW: e = std::string(f32 ? "powf(" : "pow(") + a + ", " + b + ")"; break;
      case COOT_OP_LOG10: e = std::string(f32 ? "log10f(" : "log10(") + a + ")"; break;
      case COOT_OP_SIN: e = std::string(f32 ? "sinf(" : "sin(") + a + ")"; break;
      case COOT_OP_COS: e = std::string(f32 ? "cosf(" : "cos(") + a + ")"; break;
      case COOT_OP_TAN: e = std::string(f32 ? "tanf(" : "tan(") + a + ")"; break;
      case COOT_OP_ASIN: e = std::string(f32 ? "asinf(" : "asin(") + a + ")"; break;
      case COOT_OP_ACOS: e = std::string(f32 ? "acosf(" : "acos(") + a + ")"; break;
      case COOT_OP_ATAN: e = std::string(f32 ? "atanf(" : "atan(") + a + ")"; break;
    }
    s += "  const COOT_REAL t" + std::to_string(k) + " = " + e + ";\n";
  }
  s += "  return t" + std::to_string(t.nodes.size() - 1) + ";\n}\n";
  return s;
}

const char* entry_name(const KernelSpec& spec) {
  switch (spec.kind) {
    case KIND_MAP: return spec.heads ? "coot_map_reduce" : "coot_map";
    case KIND_REDUCE: return "coot_reduce";
    case KIND_COLSUM: return "coot_colsum";
    case KIND_ROWSUM: return "coot_rowsum";
    case KIND_COLSTATS: return "coot_colstats";
    case KIND_ROWSTATS: return "coot_rowstats";
    case KIND_MULTI: return "coot_multi";
    case KIND_DIMS: return "coot_dims";
    default: return "coot_batched";
  }
}

std::string generate_source(const Tree& t, const KernelSpec& spec) {
  char pre[1024];
  std::snprintf(pre, sizeof pre,
                "// generated: tree %016" PRIx64 "\n"
                "#define COOT_ENTRY %s\n"
                "#define COOT_KIND %d\n#define COOT_NIN %d\n"
                "#define COOT_TI0 %d\n#define COOT_TI1 %d\n#define COOT_TI2 %d\n#define COOT_TI3 %d\n"
                "#define COOT_TO %d\n#define COOT_STORE %d\n#define COOT_HEADS %uu\n"
                "#define COOT_REAL %s\n#define COOT_REAL_F64 %d\n#define COOT_VEC %d\n#define COOT_UNROLL %d\n"
                "#define COOT_BLOCK %d\n#define COOT_NC %d\n",
                t.hash, entry_name(spec), spec.kind, t.n_inputs, spec.in_dtype[0], spec.in_dtype[1], spec.in_dtype[2],
                spec.in_dtype[3], spec.out_dtype, spec.store ? 1 : 0, spec.heads,
                t.compute == COOT_F32 ? "float" : "double", t.compute == COOT_F32 ? 0 : 1, spec.vec, spec.unroll,
                spec.block,
                spec.nc ? 1 : 0);
  std::string src(pre);
  if (spec.kind == KIND_MULTI || spec.kind == KIND_DIMS) {
    // several trees over the same inputs: coot_ft0 .. coot_ft3 (slots past
    // n_trees hold a constant that no code path reads), each tree's full
    // heads, whether it is stored and its storage code
    const int nt = spec.n_trees;
    char m[512];
    std::snprintf(m, sizeof m,
                  "#define COOT_NT %d\n"
                  "#define COOT_HEADS_0 %uu\n#define COOT_HEADS_1 %uu\n#define COOT_HEADS_2 %uu\n#define COOT_HEADS_3 %uu\n"
                  "#define COOT_STORE_0 %d\n#define COOT_STORE_1 %d\n#define COOT_STORE_2 %d\n#define COOT_STORE_3 %d\n"
                  "#define COOT_TO_0 %d\n#define COOT_TO_1 %d\n#define COOT_TO_2 %d\n#define COOT_TO_3 %d\n",
                  nt, spec.tree_heads[0] & COOT_HEAD_MASK, spec.tree_heads[1] & COOT_HEAD_MASK,
                  spec.tree_heads[2] & COOT_HEAD_MASK, spec.tree_heads[3] & COOT_HEAD_MASK,
                  spec.tree_out[0] >= 0, spec.tree_out[1] >= 0, spec.tree_out[2] >= 0, spec.tree_out[3] >= 0,
                  std::max(spec.tree_out[0], 0), std::max(spec.tree_out[1], 0), std::max(spec.tree_out[2], 0),
                  std::max(spec.tree_out[3], 0));
    src += m;
    if (spec.kind == KIND_DIMS) {
      // each tree's column and row sums (formed, storage code) and the
      // launch bound
      char d[512];
      std::snprintf(d, sizeof d,
                    "#define COOT_CS_0 %d\n#define COOT_CS_1 %d\n#define COOT_CS_2 %d\n#define COOT_CS_3 %d\n"
                    "#define COOT_TCS_0 %d\n#define COOT_TCS_1 %d\n#define COOT_TCS_2 %d\n#define COOT_TCS_3 %d\n"
                    "#define COOT_RS_0 %d\n#define COOT_RS_1 %d\n#define COOT_RS_2 %d\n#define COOT_RS_3 %d\n"
                    "#define COOT_TRS_0 %d\n#define COOT_TRS_1 %d\n#define COOT_TRS_2 %d\n#define COOT_TRS_3 %d\n"
                    "#define COOT_MINB %d\n#define COOT_PREFETCH %d\n",
                    spec.tree_cs[0] >= 0, spec.tree_cs[1] >= 0, spec.tree_cs[2] >= 0, spec.tree_cs[3] >= 0,
                    std::max(spec.tree_cs[0], 0), std::max(spec.tree_cs[1], 0), std::max(spec.tree_cs[2], 0),
                    std::max(spec.tree_cs[3], 0),
                    spec.tree_rs[0] >= 0, spec.tree_rs[1] >= 0, spec.tree_rs[2] >= 0, spec.tree_rs[3] >= 0,
                    std::max(spec.tree_rs[0], 0), std::max(spec.tree_rs[1], 0), std::max(spec.tree_rs[2], 0),
                    std::max(spec.tree_rs[3], 0), std::max(spec.min_blocks, 1), spec.prefetch ? 1 : 0);
      src += d;
    }
    for (int k = 0; k < 4; ++k) {
      const std::string name = "coot_ft" + std::to_string(k);
      if (k < nt && spec.trees) {
        src += tree_function(spec.trees[k], name.c_str());
      } else {
        src += "__device__ __forceinline__ COOT_REAL " + name + "(const COOT_REAL* x) { return (COOT_REAL)0; }\n";
      }
    }
  } else {
    src += tree_function(t);
  }
  src += coot_jit_rt_source;
  return src;
}

}  // namespace coot
