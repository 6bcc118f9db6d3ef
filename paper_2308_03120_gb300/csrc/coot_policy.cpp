// Learned launch shapes: features of a call, the candidate launch shapes of
// each kernel kind, and the cost model's prediction on the host.
//
// The model (a 2-layer MLP, trained on the GPU by coot_mlp.cu on timings
// the library measures itself) predicts the log of a kernel's time from
// the features of the call and of one candidate shape; the policy takes the
// candidate with the lowest prediction.  Inference runs here on the host,
// in FP64, once per distinct call (the choice is cached): a few dozen
// candidates times ~5,600 multiply-adds.
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "coot_internal.h"

namespace coot {

namespace {

std::mutex g_model_mu;
std::vector<double> g_params;  // empty: no model
int g_policy = COOT_POLICY_BUILTIN;

// candidate launch shapes {block, vec (0 = widest aligned), unroll, split
// (0 = chosen from the shape)} per kind
const int kMap[][4] = {{128, 0, 1, 0}, {128, 0, 2, 0}, {128, 0, 4, 0}, {128, 0, 8, 0},
                       {256, 0, 1, 0}, {256, 0, 2, 0}, {256, 0, 4, 0}, {256, 0, 8, 0},
                       {512, 0, 1, 0}, {512, 0, 2, 0}, {512, 0, 4, 0}, {512, 0, 8, 0}};
const int kColsum[][4] = {{128, 0, 2, 0}, {128, 0, 4, 0}, {128, 0, 8, 0}, {256, 0, 2, 0}, {256, 0, 4, 0},
                          {256, 0, 8, 0}, {128, 0, 4, 1}, {128, 0, 4, 2}, {128, 0, 4, 4}, {256, 0, 4, 1},
                          {256, 0, 4, 2}, {256, 0, 4, 4}, {256, 0, 8, 2}, {256, 0, 2, 2}};
const int kRowsum[][4] = {{256, 0, 4, 0},  {256, 0, 8, 0},  {256, 0, 16, 0}, {512, 0, 4, 0},  {512, 0, 8, 0},
                          {512, 0, 16, 0}, {256, 0, 8, 8},  {256, 0, 8, 32}, {512, 0, 8, 8},  {512, 0, 8, 16},
                          {512, 0, 8, 32}, {512, 0, 4, 8},  {512, 0, 16, 8}, {256, 0, 4, 16}};

double log2p(double x) { return std::log2(1.0 + x); }

}  // namespace

int candidates(int kind, const int (**out)[4]) {
  switch (kind) {
    case KIND_MAP:
    case KIND_REDUCE:
      *out = kMap;
      return (int)(sizeof kMap / sizeof kMap[0]);
    case KIND_COLSUM:
      *out = kColsum;
      return (int)(sizeof kColsum / sizeof kColsum[0]);
    case KIND_ROWSUM:
      *out = kRowsum;
      return (int)(sizeof kRowsum / sizeof kRowsum[0]);
  }
  *out = nullptr;
  return 0;
}

void call_features(const CallInfo& c, int block, int vec, int unroll, int64_t split, float* f) {
  int n_ops = 0, n_tr = 0;
  for (const Node& nd : c.tree->nodes) {
    if (nd.op != COOT_OP_INPUT && nd.op != COOT_OP_CONST) ++n_ops;
    if (nd.op == COOT_OP_EXP || nd.op == COOT_OP_LOG || nd.op == COOT_OP_SQRT) ++n_tr;
  }
  int heads = 0;
  for (unsigned m = c.heads; m; m &= m - 1) ++heads;
  const double n_elem = (double)c.n_rows * (double)c.n_cols;
  for (int i = 0; i < COOT_MODEL_FEATURES; ++i) f[i] = 0.f;
  // 0..4: kind (element-wise, element-wise with heads, reductions only,
  // column sums, row sums)
  int slot = 0;
  if (c.kind == KIND_MAP) slot = c.heads ? 1 : 0;
  if (c.kind == KIND_REDUCE) slot = 2;
  if (c.kind == KIND_COLSUM) slot = 3;
  if (c.kind == KIND_ROWSUM) slot = 4;
  f[slot] = 1.f;
  f[5] = (float)(log2p(n_elem) / 32.0);
  f[6] = (float)(log2p((double)c.n_rows) / 16.0);
  f[7] = (float)(log2p((double)c.n_cols) / 16.0);
  f[8] = (float)(c.tree->n_inputs / 4.0);
  f[9] = (float)(n_ops / 16.0);
  f[10] = (float)(n_tr / 8.0);
  f[11] = (float)(c.in_bytes / 8.0);
  f[12] = (float)(c.out_bytes / 8.0);
  f[13] = (float)(heads / 8.0);
  f[14] = c.dense ? 1.f : 0.f;
  f[15] = c.tree->compute == COOT_F64 ? 1.f : 0.f;
  f[16] = (float)(std::log2((double)block) / 10.0);
  f[17] = (float)(vec / 8.0);
  f[18] = (float)(std::log2((double)std::max(unroll, 1)) / 4.0);
  f[19] = (float)(log2p((double)split) / 8.0);
  f[20] = (float)(log2p(n_elem / ((double)block * std::max(vec, 1) * std::max(unroll, 1))) / 32.0);
}

bool model_ready() {
  std::lock_guard<std::mutex> lock(g_model_mu);
  return !g_params.empty();
}

int policy() {
  std::lock_guard<std::mutex> lock(g_model_mu);
  return g_policy;
}

double model_predict(const float* x) {
  const int d = COOT_MODEL_FEATURES, h = COOT_MODEL_HIDDEN;
  std::lock_guard<std::mutex> lock(g_model_mu);
  if (g_params.empty()) return 0.0;
  const double* W1 = g_params.data();
  const double* b1 = W1 + d * h;
  const double* W2 = b1 + h;
  const double* b2 = W2 + h * h;
  const double* w3 = b2 + h;
  const double b3 = w3[h];
  double h1[COOT_MODEL_HIDDEN], h2[COOT_MODEL_HIDDEN];
  for (int j = 0; j < h; ++j) {
    double s = b1[j];
    for (int i = 0; i < d; ++i) s += (double)x[i] * W1[i * h + j];
    h1[j] = s > 0.0 ? s : 0.0;
  }
  double y = b3;
  for (int j = 0; j < h; ++j) {
    double s = b2[j];
    for (int i = 0; i < h; ++i) s += h1[i] * W2[i * h + j];
    h2[j] = s > 0.0 ? s : 0.0;
    y += h2[j] * w3[j];
  }
  return y;
}

}  // namespace coot

using namespace coot;

extern "C" {

coot_status coot_model_load(const float* params, size_t n) {
  clear_error();
  // W1, b1, W2, b2, w3, b3
  const size_t want = (size_t)COOT_MODEL_FEATURES * COOT_MODEL_HIDDEN +
                      (size_t)COOT_MODEL_HIDDEN * COOT_MODEL_HIDDEN + 3 * COOT_MODEL_HIDDEN + 1;
  if (params == nullptr || n != want)
    return fail(COOT_ERR_INVALID_ARG, "model needs " + std::to_string(want) + " parameters");
  std::lock_guard<std::mutex> lock(g_model_mu);
  g_params.assign(params, params + n);
  return COOT_OK;
}

coot_status coot_model_predict(const float* features, int n_rows, float* out) {
  clear_error();
  if (!features || !out || n_rows < 0) return fail(COOT_ERR_INVALID_ARG, "bad arguments");
  if (!model_ready()) return fail(COOT_ERR_INVALID_ARG, "no model loaded");
  for (int r = 0; r < n_rows; ++r) out[r] = (float)model_predict(features + (size_t)r * COOT_MODEL_FEATURES);
  return COOT_OK;
}

coot_status coot_set_policy(int p) {
  clear_error();
  if (p != COOT_POLICY_BUILTIN && p != COOT_POLICY_LEARNED) return fail(COOT_ERR_INVALID_ARG, "unknown policy");
  if (p == COOT_POLICY_LEARNED && !model_ready()) return fail(COOT_ERR_INVALID_ARG, "no model loaded");
  std::lock_guard<std::mutex> lock(g_model_mu);
  g_policy = p;
  return COOT_OK;
}

coot_status coot_launch_candidates(int kind, int32_t* out, int max, int* n) {
  clear_error();
  const int (*c)[4] = nullptr;
  const int k = candidates(kind, &c);
  if (n) *n = k;
  if (out)
    for (int i = 0; i < k && i < max; ++i) std::memcpy(out + 4 * i, c[i], sizeof c[i]);
  return COOT_OK;
}

}  // extern "C"
