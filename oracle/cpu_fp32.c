/* FP32 evaluation of serialised expression trees on every host core: the
 * multi-core CPU side of the paper's comparison (Section 5, Task 1 times a
 * CPU library against the GPU), used as the all-cores CPU baseline of the
 * benchmark.  Test and benchmark infrastructure only: nothing in the
 * package loads it, it shares no code with the CUDA path (it decodes the
 * byte format itself), and it is not the oracle's reference arithmetic
 * (that is oracle/coot_oracle.py, in FP64).
 *
 * What it computes, for a column-major n_rows x n_cols block of FP32
 * operands (element (i, j) at in[s][i + j * ld]):
 *   out[i, j] = tree(in[0][i, j], ..., in[3][i, j]) in FP32 (C's expf,
 *               logf, sqrtf, IEEE + - * /), stored when out != NULL;
 *   heads[0..3] = sum, sum of squares, min, max of the values, summed in
 *               FP64 (NaN propagates through min / max);
 *   colsum[j] = sum of column j, rowsum[i] = sum of row i, FP64 sums
 *               rounded to FP32, when the pointers are not NULL.
 * The work is split by columns over OpenMP threads; each thread evaluates
 * a column node by node over the whole column (a vector per node, so the
 * compiler can vectorise every node), keeps its own row partials, and the
 * partials are added in thread order after the parallel region.
 *
 * Byte format (little-endian): a 16-byte header {"COOT", u16 version,
 * u16 n_nodes, u8 n_inputs, u8 compute, 6 reserved bytes}, then n_nodes
 * 16-byte nodes {u8 op, u8 0, u16 a, u16 b, u16 0, f64 imm}; the last node
 * is the root.  Only the operators of the benchmark's trees are handled:
 * input, constant, neg, abs, exp, log, sqrt, square, +, -, %, /.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OP_INPUT = 0, OP_CONST, OP_NEG, OP_ABS, OP_EXP, OP_LOG, OP_SQRT, OP_SQUARE, OP_ADD, OP_SUB, OP_MUL, OP_DIV };

typedef struct {
  int op, a, b;
  float imm;
} node_t;

static int decode(const uint8_t* buf, size_t len, node_t* nodes, int* n_nodes, int* n_inputs) {
  if (len < 16 || memcmp(buf, "COOT", 4) != 0) return -1;
  const int n = buf[6] | (buf[7] << 8);
  if (n < 1 || n > 64 || len < 16 + 16 * (size_t)n) return -1;
  *n_inputs = buf[8];
  for (int k = 0; k < n; ++k) {
    const uint8_t* p = buf + 16 + 16 * k;
    double imm;
    memcpy(&imm, p + 8, 8);
    nodes[k].op = p[0];
    nodes[k].a = p[2] | (p[3] << 8);
    nodes[k].b = p[4] | (p[5] << 8);
    nodes[k].imm = (float)imm;
    if (nodes[k].op > OP_DIV) return -2;
  }
  *n_nodes = n;
  return 0;
}

/* One column: node k's values into v + k * m (m rows). */
static void eval_column(const node_t* nodes, int n_nodes, const float* const* col, int64_t m, float* v) {
  for (int k = 0; k < n_nodes; ++k) {
    float* r = v + (int64_t)k * m;
    const node_t* nd = &nodes[k];
    const float* a = nd->op == OP_INPUT ? col[nd->a] : v + (int64_t)nd->a * m;
    const float* b = v + (int64_t)nd->b * m;
    switch (nd->op) {
      case OP_INPUT: memcpy(r, a, sizeof(float) * (size_t)m); break;
      case OP_CONST: for (int64_t i = 0; i < m; ++i) r[i] = nd->imm; break;
      case OP_NEG: for (int64_t i = 0; i < m; ++i) r[i] = -a[i]; break;
      case OP_ABS: for (int64_t i = 0; i < m; ++i) r[i] = fabsf(a[i]); break;
      case OP_EXP: for (int64_t i = 0; i < m; ++i) r[i] = expf(a[i]); break;
      case OP_LOG: for (int64_t i = 0; i < m; ++i) r[i] = logf(a[i]); break;
      case OP_SQRT: for (int64_t i = 0; i < m; ++i) r[i] = sqrtf(a[i]); break;
      case OP_SQUARE: for (int64_t i = 0; i < m; ++i) r[i] = a[i] * a[i]; break;
      case OP_ADD: for (int64_t i = 0; i < m; ++i) r[i] = a[i] + b[i]; break;
      case OP_SUB: for (int64_t i = 0; i < m; ++i) r[i] = a[i] - b[i]; break;
      case OP_MUL: for (int64_t i = 0; i < m; ++i) r[i] = a[i] * b[i]; break;
      case OP_DIV: for (int64_t i = 0; i < m; ++i) r[i] = a[i] / b[i]; break;
    }
  }
}

/* Returns 0, or a negative code for a bad tree / allocation failure.
 * threads <= 0: every core OpenMP offers. */
int cpu_fp32_eval(const uint8_t* tree, size_t len, const float* const* in, int n_in, int64_t n_rows, int64_t n_cols,
                  int64_t ld, float* out, int64_t ld_out, double* heads, float* colsum, float* rowsum, int threads) {
  node_t nodes[64];
  int n_nodes = 0, n_inputs = 0;
  const int rc = decode(tree, len, nodes, &n_nodes, &n_inputs);
  if (rc != 0) return rc;
  if (n_inputs > n_in || n_in > 4) return -3;
  int nt = 1;
#ifdef _OPENMP
  nt = threads > 0 ? threads : omp_get_max_threads();
#endif
  const int64_t m = n_rows;
  double* part = (double*)calloc((size_t)nt * (4 + (size_t)m), sizeof(double));
  float* scratch = (float*)malloc((size_t)nt * (size_t)n_nodes * (size_t)(m > 0 ? m : 1) * sizeof(float));
  if (!part || !scratch) {
    free(part);
    free(scratch);
    return -4;
  }
  for (int t = 0; t < nt; ++t) {
    part[(size_t)t * (4 + m) + 2] = INFINITY;
    part[(size_t)t * (4 + m) + 3] = -INFINITY;
  }
#pragma omp parallel num_threads(nt)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    double* h = part + (size_t)t * (4 + m);
    double* rows = h + 4;
    float* v = scratch + (size_t)t * (size_t)n_nodes * (size_t)(m > 0 ? m : 1);
    const float* col[4] = {0, 0, 0, 0};
#pragma omp for schedule(static)
    for (int64_t j = 0; j < n_cols; ++j) {
      for (int s = 0; s < n_in; ++s) col[s] = in[s] + j * ld;
      eval_column(nodes, n_nodes, col, m, v);
      const float* y = v + (int64_t)(n_nodes - 1) * m;
      if (out) memcpy(out + j * ld_out, y, sizeof(float) * (size_t)m);
      double cs = 0.0;
      for (int64_t i = 0; i < m; ++i) {
        const double d = (double)y[i];
        cs += d;
        h[1] += d * d;
        rows[i] += d;
        if (!(d >= h[2])) h[2] = (d != d || h[2] != h[2]) ? NAN : d;
        if (!(d <= h[3])) h[3] = (d != d || h[3] != h[3]) ? NAN : d;
      }
      h[0] += cs;
      if (colsum) colsum[j] = (float)cs;
    }
  }
  if (heads) {
    heads[0] = heads[1] = 0.0;
    heads[2] = INFINITY;
    heads[3] = -INFINITY;
  }
  for (int t = 0; t < nt; ++t) {
    const double* h = part + (size_t)t * (4 + m);
    if (heads) {
      heads[0] += h[0];
      heads[1] += h[1];
      heads[2] = (h[2] != h[2] || heads[2] != heads[2]) ? NAN : fmin(heads[2], h[2]);
      heads[3] = (h[3] != h[3] || heads[3] != heads[3]) ? NAN : fmax(heads[3], h[3]);
    }
  }
  if (rowsum) {
    for (int64_t i = 0; i < m; ++i) {
      double s = 0.0;
      for (int t = 0; t < nt; ++t) s += part[(size_t)t * (4 + m) + 4 + i];
      rowsum[i] = (float)s;
    }
  }
  free(part);
  free(scratch);
  return 0;
}

/* Threads the evaluator uses by default. */
int cpu_fp32_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
