// Canonical form of an expression tree: exact rewrites applied before a
// kernel is generated, in the spirit of the compile-time rewrites that
// Bandicoot's expression types make while an expression is being built
// (Section 7: trans(diagmat(V)) returns the diagmat unchanged).
//
// Every rewrite gives the same IEEE result for every input (NaN payloads
// aside), so a canonical tree is evaluated exactly as the original:
//   * common subexpressions become one node, nodes the root does not use
//     are dropped, and commutative nodes (+, %, ==, !=) put a constant
//     operand first so that x * 2 and 2 * x are the same node;
//   * constant subtrees of exactly rounded operations (+ - % / neg abs
//     square sqrt and the relations) are folded in the compute type;
//     exp / log / pow / trig are left alone (the host's library is not the
//     device's);
//   * sign rules: -(-x) = x, |-x| = |x|, ||x|| = |x|, (-x)^2 = |x|^2 = x^2,
//     x + (-y) = x - y, (-x) + y = y - x, x - (-y) = x + y,
//     (-x) % (-y) = x % y, (-x) / (-y) = x / y, -(k % x) = (-k) % x,
//     k % (-x) = (-k) % x;
//   * identities: x % 1 = x / 1 = x, x % -1 = x / -1 = -x, x - 0 = x,
//     x + (-0) = x (x + 0 is kept: it turns -0 into +0);
//   * scalar merging: k1 % (k2 % x) = (k1 k2) % x when k1 and k2 are powers
//     of two of magnitude at least 1 (the product scales x exactly, and an
//     intermediate overflow implies the merged one);
//   * input slots that name the same matrix in a call become one slot, and
//     slots the tree does not read are dropped: the kernel reads each
//     distinct operand once (dot(x, x) reads x once).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "coot_internal.h"

namespace coot {

namespace {

thread_local bool g_canonical = true;

bool is_unary_op(int op) {
  return (op >= COOT_OP_NEG && op <= COOT_OP_SQUARE) || (op >= COOT_OP_LOG10 && op <= COOT_OP_ATAN);
}
bool is_binary_op(int op) { return op >= COOT_OP_ADD && op <= COOT_OP_POW; }


struct Builder {
  const Tree& src;
  const int* slot_alias;  // representative slot of each input slot, or null
  std::vector<Node> nodes;
  std::map<std::tuple<int, int, int, uint64_t>, int> seen;
  std::vector<int> memo;

  Builder(const Tree& t, const int* alias) : src(t), slot_alias(alias), memo(t.nodes.size(), -1) {}

  bool f32() const { return src.compute == COOT_F32; }
  double round(double v) const { return f32() ? (double)(float)v : v; }

  int add(uint8_t op, int a, int b, double imm) {
    uint64_t bits = 0;
    if (op == COOT_OP_CONST) std::memcpy(&bits, &imm, 8);
    const auto key = std::make_tuple((int)op, a, b, bits);
    auto it = seen.find(key);
    if (it != seen.end()) return it->second;
    Node n;
    n.op = op;
    n.a = (uint16_t)a;
    n.b = (uint16_t)b;
    n.imm = op == COOT_OP_CONST ? imm : 0.0;
    nodes.push_back(n);
    seen.emplace(key, (int)nodes.size() - 1);
    return (int)nodes.size() - 1;
  }

  bool is_const(int k) const { return nodes[k].op == COOT_OP_CONST; }
  double cval(int k) const { return nodes[k].imm; }
  bool is(int k, int op) const { return nodes[k].op == op; }

  int constant(double v) { return add(COOT_OP_CONST, 0, 0, round(v)); }

  // one exactly rounded operation on constants, in the compute type
  double fold1(int op, double x) const {
    if (f32()) {
      const float a = (float)x;
      switch (op) {
        case COOT_OP_NEG: return -a;
        case COOT_OP_ABS: return std::fabs(a);
        case COOT_OP_SQUARE: { const float r = a * a; return r; }
        default: return std::sqrt(a);
      }
    }
    switch (op) {
      case COOT_OP_NEG: return -x;
      case COOT_OP_ABS: return std::fabs(x);
      case COOT_OP_SQUARE: { const double r = x * x; return r; }
      default: return std::sqrt(x);
    }
  }
  double fold2(int op, double x, double y) const {
    if (f32()) {
      const float a = (float)x, b = (float)y;
      switch (op) {
        case COOT_OP_ADD: { const float r = a + b; return r; }
        case COOT_OP_SUB: { const float r = a - b; return r; }
        case COOT_OP_MUL: { const float r = a * b; return r; }
        case COOT_OP_DIV: { const float r = a / b; return r; }
        case COOT_OP_LT: return a < b ? 1.0 : 0.0;
        case COOT_OP_LE: return a <= b ? 1.0 : 0.0;
        case COOT_OP_GT: return a > b ? 1.0 : 0.0;
        case COOT_OP_GE: return a >= b ? 1.0 : 0.0;
        case COOT_OP_EQ: return a == b ? 1.0 : 0.0;
        default: return a != b ? 1.0 : 0.0;
      }
    }
    switch (op) {
      case COOT_OP_ADD: { const double r = x + y; return r; }
      case COOT_OP_SUB: { const double r = x - y; return r; }
      case COOT_OP_MUL: { const double r = x * y; return r; }
      case COOT_OP_DIV: { const double r = x / y; return r; }
      case COOT_OP_LT: return x < y ? 1.0 : 0.0;
      case COOT_OP_LE: return x <= y ? 1.0 : 0.0;
      case COOT_OP_GT: return x > y ? 1.0 : 0.0;
      case COOT_OP_GE: return x >= y ? 1.0 : 0.0;
      case COOT_OP_EQ: return x == y ? 1.0 : 0.0;
      default: return x != y ? 1.0 : 0.0;
    }
  }

  static bool pow2_ge1(double v) {
    if (!(std::fabs(v) >= 1.0) || !std::isfinite(v)) return false;
    int e = 0;
    return std::fabs(std::frexp(v, &e)) == 0.5;
  }

  int unary(int op, int a) {
    const bool foldable = op == COOT_OP_NEG || op == COOT_OP_ABS || op == COOT_OP_SQUARE || op == COOT_OP_SQRT;
    if (foldable && is_const(a)) return constant(fold1(op, cval(a)));
    switch (op) {
      case COOT_OP_NEG:
        if (is(a, COOT_OP_NEG)) return nodes[a].a;
        if (is(a, COOT_OP_MUL) && is_const(nodes[a].a))
          return mul(constant(-cval(nodes[a].a)), nodes[a].b);
        break;
      case COOT_OP_ABS:
        if (is(a, COOT_OP_NEG)) return unary(COOT_OP_ABS, nodes[a].a);
        if (is(a, COOT_OP_ABS)) return a;
        break;
      case COOT_OP_SQUARE:
        if (is(a, COOT_OP_NEG) || is(a, COOT_OP_ABS)) return unary(COOT_OP_SQUARE, nodes[a].a);
        break;
      default:
        break;
    }
    return add((uint8_t)op, a, 0, 0.0);
  }

  int mul(int a, int b) {
    if (is_const(b) && !is_const(a)) std::swap(a, b);  // constant first
    if (is_const(a) && is_const(b)) return constant(fold2(COOT_OP_MUL, cval(a), cval(b)));
    if (is_const(a)) {
      const double k = cval(a);
      if (k == 1.0) return b;
      if (k == -1.0) return unary(COOT_OP_NEG, b);
      if (is(b, COOT_OP_NEG)) return mul(constant(-k), nodes[b].a);
      if (is(b, COOT_OP_MUL) && is_const(nodes[b].a) && pow2_ge1(k) && pow2_ge1(cval(nodes[b].a)) &&
          std::isfinite(round(k * cval(nodes[b].a))))
        return mul(constant(k * cval(nodes[b].a)), nodes[b].b);
    }
    if (is(a, COOT_OP_NEG) && is(b, COOT_OP_NEG)) return mul(nodes[a].a, nodes[b].a);
    return add(COOT_OP_MUL, a, b, 0.0);
  }

  int binary(int op, int a, int b) {
    const bool foldable = op == COOT_OP_ADD || op == COOT_OP_SUB || op == COOT_OP_MUL || op == COOT_OP_DIV ||
                          (op >= COOT_OP_LT && op <= COOT_OP_NE);
    if (foldable && is_const(a) && is_const(b)) return constant(fold2(op, cval(a), cval(b)));
    switch (op) {
      case COOT_OP_MUL:
        return mul(a, b);
      case COOT_OP_ADD:
        if (is_const(b) && !is_const(a)) std::swap(a, b);
        if (is_const(a) && cval(a) == 0.0 && std::signbit(cval(a))) return b;  // (-0) + x = x
        if (is(b, COOT_OP_NEG)) return binary(COOT_OP_SUB, a, nodes[b].a);
        if (is(a, COOT_OP_NEG)) return binary(COOT_OP_SUB, b, nodes[a].a);
        break;
      case COOT_OP_SUB:
        if (is_const(b) && cval(b) == 0.0 && !std::signbit(cval(b))) return a;  // x - 0 = x
        if (is(b, COOT_OP_NEG)) return binary(COOT_OP_ADD, a, nodes[b].a);
        break;
      case COOT_OP_DIV:
        if (is_const(b) && cval(b) == 1.0) return a;
        if (is_const(b) && cval(b) == -1.0) return unary(COOT_OP_NEG, a);
        if (is(a, COOT_OP_NEG) && is(b, COOT_OP_NEG)) return binary(COOT_OP_DIV, nodes[a].a, nodes[b].a);
        break;
      case COOT_OP_EQ:
      case COOT_OP_NE:
        if (is_const(b) && !is_const(a)) std::swap(a, b);
        break;
      default:
        break;
    }
    return add((uint8_t)op, a, b, 0.0);
  }

  int build(int k) {
    if (memo[k] >= 0) return memo[k];
    const Node& n = src.nodes[k];
    int r;
    if (n.op == COOT_OP_INPUT) {
      r = add(COOT_OP_INPUT, slot_alias ? slot_alias[n.a] : n.a, 0, 0.0);
    } else if (n.op == COOT_OP_CONST) {
      r = constant(n.imm);
    } else if (is_unary_op(n.op)) {
      r = unary(n.op, build(n.a));
    } else {
      const int a = build(n.a);
      r = binary(n.op, a, build(n.b));
    }
    memo[k] = r;
    return r;
  }
};

// the nodes reachable from k, operands first (at most 64 nodes deep)
void reachable(const std::vector<Node>& nodes, int k, std::vector<int>* order, std::vector<int>* index) {
  if ((*index)[k] >= 0) return;
  const Node& n = nodes[k];
  if (is_unary_op(n.op) || is_binary_op(n.op)) reachable(nodes, n.a, order, index);
  if (is_binary_op(n.op)) reachable(nodes, n.b, order, index);
  (*index)[k] = (int)order->size();
  order->push_back(k);
}

}  // namespace

bool canonical_enabled() { return g_canonical; }
void set_canonical(bool on) { g_canonical = on; }

void canonicalize(const Tree& in, const int* slot_alias, Tree* out, std::vector<int>* kept_slots, bool keep_slots) {
  Builder b(in, slot_alias);
  const int root = b.build((int)in.nodes.size() - 1);
  // keep what the root reaches, operands first
  std::vector<int> order, index(b.nodes.size(), -1);
  reachable(b.nodes, root, &order, &index);
  // input slots the tree reads, renumbered in slot order
  std::vector<int> used;
  for (int k : order)
    if (b.nodes[k].op == COOT_OP_INPUT) used.push_back(b.nodes[k].a);
  std::sort(used.begin(), used.end());
  used.erase(std::unique(used.begin(), used.end()), used.end());
  if (used.empty()) used.push_back(0);  // a constant tree keeps slot 0 for its shape
  if (keep_slots) {
    used.clear();
    for (int i = 0; i < in.n_inputs; ++i) used.push_back(i);
  }
  Tree t;
  t.compute = in.compute;
  t.n_inputs = (int)used.size();
  for (int k : order) {
    Node n = b.nodes[k];
    if (n.op == COOT_OP_INPUT) {
      n.a = (uint16_t)(std::lower_bound(used.begin(), used.end(), (int)n.a) - used.begin());
    } else if (n.op != COOT_OP_CONST) {
      n.a = (uint16_t)index[n.a];
      n.b = is_binary_op(n.op) ? (uint16_t)index[n.b] : 0;
    }
    t.nodes.push_back(n);
  }
  // the cache key of the canonical form
  uint64_t h = fnv1a("canon", 5);
  h = fnv1a(&t.compute, sizeof t.compute, h);
  h = fnv1a(&t.n_inputs, sizeof t.n_inputs, h);
  for (const Node& n : t.nodes) {
    h = fnv1a(&n.op, 1, h);
    h = fnv1a(&n.a, 2, h);
    h = fnv1a(&n.b, 2, h);
    h = fnv1a(&n.imm, 8, h);
  }
  t.hash = h;
  if (kept_slots) *kept_slots = used;
  *out = std::move(t);
}

// Serialised form of a tree (the byte layout of coot.h).
std::vector<uint8_t> serialise(const Tree& t) {
  std::vector<uint8_t> buf(16 + 16 * t.nodes.size(), 0);
  std::memcpy(buf.data(), "COOT", 4);
  buf[4] = 1;
  buf[6] = (uint8_t)(t.nodes.size() & 0xff);
  buf[7] = (uint8_t)(t.nodes.size() >> 8);
  buf[8] = (uint8_t)t.n_inputs;
  buf[9] = (uint8_t)t.compute;
  for (size_t k = 0; k < t.nodes.size(); ++k) {
    uint8_t* p = buf.data() + 16 + 16 * k;
    const Node& n = t.nodes[k];
    p[0] = n.op;
    p[2] = (uint8_t)(n.a & 0xff);
    p[3] = (uint8_t)(n.a >> 8);
    p[4] = (uint8_t)(n.b & 0xff);
    p[5] = (uint8_t)(n.b >> 8);
    uint64_t u;
    std::memcpy(&u, &n.imm, 8);
    for (int i = 0; i < 8; ++i) p[8 + i] = (uint8_t)(u >> (8 * i));
  }
  return buf;
}

}  // namespace coot

using namespace coot;

extern "C" {

coot_status coot_set_canonical(int enable) {
  clear_error();
  set_canonical(enable != 0);
  return COOT_OK;
}

coot_status coot_tree_canonical(const uint8_t* tree, size_t len, uint8_t* out, size_t cap, size_t* out_len) {
  clear_error();
  Tree t;
  coot_status s = parse_tree(tree, len, &t);
  if (s != COOT_OK) return s;
  Tree c;
  canonicalize(t, nullptr, &c, nullptr, true);
  const std::vector<uint8_t> bytes = serialise(c);
  if (out_len) *out_len = bytes.size();
  if (out && cap) std::memcpy(out, bytes.data(), std::min(cap, bytes.size()));
  return COOT_OK;
}

}  // extern "C"
