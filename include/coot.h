/*
 * coot.h - C ABI of the fused expression + reduction engine for GB300
 * (sm_103a).
 *
 * The engine evaluates element-wise expression trees over column-major
 * matrices and vectors in ONE fused GPU kernel per call, without
 * temporaries, and can feed the element values straight into reductions.
 * It implements the evaluation model of Bandicoot (Curtin, Edel, Sanderson,
 * arXiv 2308.03120):
 *   - expressions are trees of element-wise nodes (the paper's eOp / eGlue
 *     expression types, Section 7) built from the operators of Table 2 and
 *     the element-wise functions of Table 7;
 *   - evaluation is delayed until the result is assigned (Section 7,
 *     "operator="): the caller hands the whole tree over in one call;
 *   - the reductions are those of Table 5 (accu, dot, norm) and Table 6
 *     (sum / min / max along a dimension);
 *   - matrices are column-major ("(i)" walks column by column, Table 1).
 * Where the paper evaluates each tree node with at least one kernel launch
 * (Section 7: it cannot generate code per expression), this library
 * generates and compiles one kernel per tree at run time (cached).
 *
 * Memory and ownership.  Every pointer in a coot_mat, every result pointer
 * (`out_dev`), every workspace (`ws`) and every stream belongs to the
 * caller; the library never allocates or frees them.  Matrix and result
 * pointers are DEVICE pointers unless a function says otherwise.  The
 * library owns only its compiled-kernel cache.
 *
 * Asynchrony.  Calls enqueue work on `stream` (a cudaStream_t; NULL = the
 * legacy default stream) and return without waiting.  Results are valid
 * once the stream has reached the call (cudaStreamSynchronize or an event).
 * Host-side checks happen before anything is enqueued: on any error status
 * nothing has been enqueued and no output has been written.
 *
 * Errors.  Every function returns a coot_status; nothing throws across the
 * ABI.  coot_last_error() returns a message for the most recent failing
 * call on the calling thread.  A CUDA error raised by a launch is returned
 * as COOT_ERR_CUDA.
 *
 * Workspace.  Reductions need a small scratch area (`ws`, `ws_bytes`) for
 * per-block partial results and arrival counters.  coot_workspace_size()
 * gives a size that suffices for every call on operands of up to a given
 * row count; a call checks `ws_bytes` and picks a launch shape that fits,
 * or returns COOT_ERR_WORKSPACE.  The caller allocates the workspace on the
 * device and ZERO-FILLS it once before its first use.  Every call that
 * completes leaves the counters at zero again, so the same workspace can be
 * reused by later calls on the same stream.  Two calls that run
 * concurrently (different streams) need different workspaces.
 *
 * Aliasing.  An element-wise output may be exactly one of the inputs (same
 * pointer, shape, dtype and ld): every element is read before it is written
 * by the same thread, so "B = B + 3 * A" (the paper's Task 2, B += 3 * A) is
 * valid.  Any other overlap between the output and an input is rejected
 * with COOT_ERR_ALIAS.
 */
#ifndef COOT_H
#define COOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum coot_status {
  COOT_OK = 0,
  COOT_ERR_INVALID_ARG = 1, /* null pointer, bad enum value, negative size   */
  COOT_ERR_BAD_TREE = 2,    /* malformed serialised tree                      */
  COOT_ERR_SHAPE = 3,       /* operand / output shapes do not conform         */
  COOT_ERR_DTYPE = 4,       /* unsupported storage type for this operand      */
  COOT_ERR_ALIAS = 5,       /* output partially overlaps an input             */
  COOT_ERR_EMPTY = 6,       /* min/max of an object with no elements          */
  COOT_ERR_UNSUPPORTED = 7, /* valid request this library does not implement  */
  COOT_ERR_COMPILE = 8,     /* run-time compilation of a kernel failed        */
  COOT_ERR_CUDA = 9,        /* a CUDA runtime call or a launch failed         */
  COOT_ERR_TIMEOUT = 10,    /* a bounded device-side wait gave up             */
  COOT_ERR_NOT_INIT = 11,   /* coot_init has not been called                  */
  COOT_ERR_WORKSPACE = 12   /* workspace missing or too small                 */
} coot_status;

/* Storage types.  Arithmetic happens in the tree's compute type (FP32 or
 * FP64); BF16 / FP16 elements are widened exactly on load and rounded to
 * nearest-even on store (the paper's fused conversion, Section 7). */
typedef enum coot_dtype {
  COOT_F32 = 0,
  COOT_BF16 = 1,
  COOT_F16 = 2,
  COOT_F64 = 3,
  /* Integer storage (Section 7's conversion example reads an integer matrix
   * into a float expression): converted to the compute type on load (to
   * the nearest FP32 for an FP32 tree, exact up to 2^24; exact in FP64).
   * As element-wise outputs they receive the value rounded toward zero,
   * saturated to the type's range, NaN stored as 0.  Sums, statistics and
   * column sums are not stored in integer types. */
  COOT_I32 = 4,
  COOT_U32 = 5
} coot_dtype;

/* A column-major matrix in device memory: element (i, j), 0 <= i < n_rows,
 * 0 <= j < n_cols, lives at ((T*)ptr)[i + j * ld] with T the storage type.
 * ld >= max(n_rows, 1).  A vector is an n x 1 (column) or 1 x n (row)
 * matrix (Table 1, Col / Row).  n_rows * n_cols == 0 is an empty object.
 * ptr may also be the device address of pinned host memory
 * (coot_host_device_pointer): the kernels then read or write that memory
 * directly. */
typedef struct coot_mat {
  void* ptr;
  int32_t dtype; /* coot_dtype */
  int32_t reserved; /* must be 0 */
  int64_t n_rows;
  int64_t n_cols;
  int64_t ld;
} coot_mat;

/* ------------------------------------------------------------------------
 * Serialised expression tree (little-endian), the run-time form of the
 * paper's expression types (eOp / eGlue, Section 7):
 *
 *   header, 16 bytes:
 *     char     magic[4] = "COOT"
 *     uint16_t version = 1
 *     uint16_t n_nodes        1..64
 *     uint8_t  n_inputs       1..4   number of input slots (operands passed)
 *     uint8_t  compute        0 = FP32, 3 = FP64 arithmetic
 *     uint16_t reserved = 0
 *     uint32_t reserved = 0
 *   node k (k = 0 .. n_nodes-1), 16 bytes at offset 16 + 16 k:
 *     uint8_t  op             a coot_op below
 *     uint8_t  reserved = 0
 *     uint16_t a              operand: an earlier node (a < k) or, for
 *                             COOT_OP_INPUT, the input slot (< n_inputs)
 *     uint16_t b              second operand of binary nodes (b < k), else 0
 *     uint16_t reserved = 0
 *     double   imm            value of COOT_OP_CONST, else ignored (write 0)
 *
 * The last node is the root.  Nodes may be shared (a DAG).  Immediates are
 * rounded to the compute type before use.  Scalar forms of Table 2
 * ("A + k", "k - A", "A * k", ...) are binary nodes with a constant operand.
 * ---------------------------------------------------------------------- */
typedef enum coot_op {
  COOT_OP_INPUT = 0,  /* input slot a                                      */
  COOT_OP_CONST = 1,  /* scalar imm                                        */
  COOT_OP_NEG = 2,    /* -a                                                */
  COOT_OP_ABS = 3,    /* |a|                                               */
  COOT_OP_EXP = 4,    /* exp(a)      Table 7                               */
  COOT_OP_LOG = 5,    /* log(a)      Table 7 (natural logarithm)           */
  COOT_OP_SQRT = 6,   /* sqrt(a)     Table 7                               */
  COOT_OP_SQUARE = 7, /* a * a       Table 7                               */
  COOT_OP_ADD = 8,    /* a + b       Table 2                               */
  COOT_OP_SUB = 9,    /* a - b       Table 2                               */
  COOT_OP_MUL = 10,   /* a % b       Table 2, element-wise (Schur) product */
  COOT_OP_DIV = 11,   /* a / b       Table 2, element-wise division        */
  /* Relational operators (the "A < x" of Table 5's all/any rows, "other
   * relational expressions may also be used"): 1 where the relation holds,
   * else 0, in the compute type.  NaN is unordered: every relation with a
   * NaN operand is false except COOT_OP_NE. */
  COOT_OP_LT = 12,    /* a < b                                             */
  COOT_OP_LE = 13,    /* a <= b                                            */
  COOT_OP_GT = 14,    /* a > b                                             */
  COOT_OP_GE = 15,    /* a >= b                                            */
  COOT_OP_EQ = 16,    /* a == b                                            */
  COOT_OP_NE = 17,    /* a != b                                            */
  /* Table 7: pow and log10 ("misc(A)") and the trigonometric functions
   * ("trig(A)"), in the compute type's CUDA functions (no fast maths; pow
   * follows C's pow for the special cases). */
  COOT_OP_POW = 18,   /* pow(a, b)                                         */
  COOT_OP_LOG10 = 19, /* log10(a)                                          */
  COOT_OP_SIN = 20,   /* sin(a)                                            */
  COOT_OP_COS = 21,   /* cos(a)                                            */
  COOT_OP_TAN = 22,   /* tan(a)                                            */
  COOT_OP_ASIN = 23,  /* asin(a)                                           */
  COOT_OP_ACOS = 24,  /* acos(a)                                           */
  COOT_OP_ATAN = 25   /* atan(a)                                           */
} coot_op;

#define COOT_TREE_MAX_NODES 64
#define COOT_TREE_MAX_INPUTS 4

/* Reduction heads for coot_expr_reduce: one result per set bit, written to
 * out_dev[] in increasing bit order, as FP64. */
#define COOT_HEAD_SUM    (1u << 0) /* sum of all elements (accu, Table 5)     */
#define COOT_HEAD_SUMSQ  (1u << 1) /* sum of squares                           */
#define COOT_HEAD_NORM2  (1u << 2) /* sqrt(sum of squares) (norm "fro" / 2)    */
#define COOT_HEAD_SUMABS (1u << 3) /* sum of magnitudes (vector norm p = 1)    */
#define COOT_HEAD_MIN    (1u << 4) /* smallest element (NaN propagates)        */
#define COOT_HEAD_MAX    (1u << 5) /* largest element (NaN propagates)         */
#define COOT_HEAD_MINABS (1u << 6) /* smallest magnitude (norm p = "-inf")     */
#define COOT_HEAD_MAXABS (1u << 7) /* largest magnitude (norm p = "inf")       */
#define COOT_HEAD_ALL    (1u << 8) /* 1 if every element is nonzero, else 0
                                      (all, Table 5; NaN is nonzero; 1 when
                                      there are no elements)                 */
#define COOT_HEAD_ANY    (1u << 9) /* 1 if some element is nonzero, else 0
                                      (any, Table 5; 0 when there are none)  */
#define COOT_HEAD_MASK   0x3FFu    /* every head bit                          */
/* Sums along a dimension, formed in the same pass (coot_expr_multi_dims
 * only; they write matrices, not out_dev entries): */
#define COOT_HEAD_COLSUM (1u << 10) /* sum(A, 0), each column's sum (Table 6) */
#define COOT_HEAD_ROWSUM (1u << 11) /* sum(A, 1), each row's sum (Table 6)    */

/* norm(A, p) selectors (Table 5): p = 1, 2, or one of these. */
#define COOT_NORM_INF (-1)
#define COOT_NORM_NEG_INF (-2)
#define COOT_NORM_FRO (-3)

/* ------------------------------------------------------------------------
 * Set-up
 * ---------------------------------------------------------------------- */

/* Select `device` (cudaSetDevice) and prepare the kernel cache; cf. the
 * paper's coot_init(backend, print_info, device) (Section 2).  flags: bit 0
 * = print device information to stderr.  Safe to call again; returns
 * COOT_ERR_CUDA if the device cannot be used. */
coot_status coot_init(int device, unsigned flags);

/* Drop every cached kernel module (not the on-disk cache). */
coot_status coot_finalize(void);

/* Message for the last failing call on this thread ("" if none).  The
 * pointer stays valid until the next call on this thread. */
const char* coot_last_error(void);

/* Short name of a status code. */
const char* coot_status_string(coot_status s);

/* Library version as MAJOR * 10000 + MINOR * 100 + PATCH. */
int coot_version(void);

/* Bytes of workspace that suffice for every call on operands with at most
 * `max_rows` rows (any number of columns).  Host-only. */
coot_status coot_workspace_size(int64_t max_rows, size_t* bytes);

/* Launch shape of the kernels of one kind (0 element-wise / with heads,
 * 1 reductions only, 2 column sums, 3 row sums, 4 batched, 5 column
 * statistics, 6 row statistics, 7 several trees in one pass; row
 * statistics use at most 256 threads per block; 8 several trees with sums
 * along a dimension, where unroll is the vectors per lane in a row segment
 * and split the number of column chunks) for the calls
 * that follow ON THIS THREAD, for tuning and for the learned selection of
 * launch shapes (not in the paper).  block: threads per block, 64..1024 in
 * steps of 64, or 0 to drop the setting (back to the built-in choice);
 * vec: elements per vector access (1, 2, 4, 8; 0 = widest the operands'
 * alignment allows; a width they do not allow is lowered); unroll: vector
 * accesses in flight per thread and input, 1..16 (0 = built-in); for the
 * batched kind, `block` counts the computing threads (one staging warp is
 * added to each block, up to 992 + 32) and `unroll` the rows in flight per
 * lane of a unit read from global memory; blocks_per_sm: cap on resident
 * blocks per SM for the persistent grid (0 = occupancy limit); split:
 * column sums and statistics: segments per column, row sums and
 * statistics: column chunks (0 =
 * chosen from the shape; capped by the workspace).  Host-only. */
coot_status coot_set_launch_config(int kind, int block, int vec, int unroll, int blocks_per_sm,
                                   int64_t split);

/* Compile and load (without launching) the kernel a call of this kind
 * would use with exactly this launch shape (vec 1/2/4/8, unroll 1..16):
 * first-use compilation moves out of timed regions and graph captures.
 * dtypes: host array of the tree's input storage types; out_dtype: -1 when
 * nothing element-wise is stored.  Kinds 0..6; the several-tree kernel
 * (kind 7) is compiled by its first coot_expr_multi call
 * (COOT_ERR_UNSUPPORTED).  Thread-safe; threads compile in parallel.
 * Needs coot_init. */
coot_status coot_prepare(const uint8_t* tree, size_t tree_len, int kind, const int32_t* dtypes,
                         int out_dtype, unsigned heads, int block, int vec, int unroll);

/* Launch shape of the last kernel launched by a coot call on this thread
 * (any out pointer may be NULL).  Host-only. */
coot_status coot_last_launch(int* block, int* vec, int* unroll, int64_t* grid, int64_t* split);

/* Canonical form (on by default, per thread): before a call generates its
 * kernel, its tree is rewritten with exact rules only -- shared
 * subexpressions merged, unused nodes dropped, constant subtrees of exactly
 * rounded operations folded in the compute type, sign and identity rules
 * (-(-x) = x, x + (-y) = x - y, x % 1 = x, ...), scalar multiples by powers
 * of two >= 1 merged -- and input slots that name the same matrix, or that
 * the tree does not read, are merged or dropped, so every distinct operand
 * is read once.  The result is the same value for every input (the
 * compile-time rewrites of Section 7, at run time).  enable = 0 turns it off
 * for the calls that follow on this thread (for measurement).  Host-only. */
coot_status coot_set_canonical(int enable);

/* The canonical form of a tree into out (cap bytes; the full length goes to
 * *out_len).  Input slots keep their numbers (the merging and dropping of
 * slots happens per call, where the operands are known).  Host-only. */
coot_status coot_tree_canonical(const uint8_t* tree, size_t tree_len, uint8_t* out, size_t cap,
                                size_t* out_len);

/* Validate a serialised tree without a GPU: on success *n_inputs receives
 * the tree's input count, *compute its compute dtype (COOT_F32 or COOT_F64)
 * and *hash a 64-bit FNV-1a digest of the bytes (the kernel-cache key).
 * Any of the out pointers may be NULL.  Host-only. */
coot_status coot_tree_check(const uint8_t* tree, size_t tree_len, int* n_inputs,
                            int* compute, uint64_t* hash);

/* Compile the kernel of a tree with NVRTC for `arch` (e.g. "sm_103a")
 * without loading it (no GPU needed); *cubin_bytes receives the size of
 * the result.  kind as for coot_tree_source; in_dtype / out_dtype are the
 * storage types of every input and of the output; heads as for
 * coot_expr_reduce.  Host-only; for build checks and tests. */
coot_status coot_tree_compile(const uint8_t* tree, size_t tree_len, int kind, int in_dtype,
                              int out_dtype, unsigned heads, const char* arch,
                              size_t* cubin_bytes);

/* Write the CUDA source generated for a tree into buf (NUL-terminated,
 * truncated to buf_len) and its full length to *len.  kind: 0 = element-wise
 * evaluation, 1 = full reduction, 2 = column sums, 3 = row sums,
 * 4 = batched evaluation, 5 / 6 = column / row statistics (all six),
 * 7 = the several-tree kernel with this one tree, 8 = the same with its
 * column and row sums (coot_tree_compile: those of the COOT_HEAD_COLSUM /
 * COOT_HEAD_ROWSUM bits of `heads`, both when neither is set); every input
 * and the output FP32.  Host-only;
 * for inspection and tests. */
coot_status coot_tree_source(const uint8_t* tree, size_t tree_len, int kind, char* buf,
                             size_t buf_len, size_t* len);

/* ------------------------------------------------------------------------
 * Evaluation.  `tree`/`tree_len` are a host buffer with the serialised
 * tree; `in` is a host array of n_in device matrices (n_in == the tree's
 * n_inputs), all with the same n_rows and n_cols (element-wise operations
 * need equal sizes, Table 2).
 * ---------------------------------------------------------------------- */

/* out = tree(in...) element by element (delayed evaluation at assignment,
 * Section 7; fused type conversion into out's storage type).  out must have
 * the inputs' shape.  Empty shapes are a no-op. */
coot_status coot_expr_eval(const uint8_t* tree, size_t tree_len, const coot_mat* in, int n_in,
                           const coot_mat* out, void* ws, size_t ws_bytes, void* stream);

/* out_dev[0] = accu(tree(in...)) = sum of all elements (Table 5), FP64.
 * Empty -> 0. */
coot_status coot_accu(const uint8_t* tree, size_t tree_len, const coot_mat* in, int n_in,
                      double* out_dev, void* ws, size_t ws_bytes, void* stream);

/* sum(tree(in...), dim) (Table 6): dim = 0 -> the sum of each column, out
 * is 1 x n_cols; dim = 1 -> the sum of each row, out is n_rows x 1.  out may
 * be any storage type (sums are formed in FP64 across blocks and rounded
 * once).  out must not overlap an input. */
coot_status coot_sum_dim(const uint8_t* tree, size_t tree_len, const coot_mat* in, int n_in,
                         int dim, const coot_mat* out, void* ws, size_t ws_bytes, void* stream);

/* out_dev[0] = dot(a, b) = sum_i a_i * b_i over column-major element order;
 * a and b need equal element counts, not equal shapes (Table 5).  FP32
 * products (FP64 if either operand is FP64). */
coot_status coot_dot(const coot_mat* a, const coot_mat* b, double* out_dev, void* ws,
                     size_t ws_bytes, void* stream);

/* out_dev[0] = norm(tree(in...), p) (Table 5).  p = 2 on a vector or
 * COOT_NORM_FRO on anything: sqrt of the sum of squares; p = 1: sum of
 * magnitudes; COOT_NORM_INF / COOT_NORM_NEG_INF: largest / smallest
 * magnitude (vectors).  p = 2 of a matrix is the spectral norm and returns
 * COOT_ERR_UNSUPPORTED.  Empty -> 0. */
coot_status coot_norm(const uint8_t* tree, size_t tree_len, const coot_mat* in, int n_in, int p,
                      double* out_dev, void* ws, size_t ws_bytes, void* stream);

/* out_dev[0] = all(tree(in...)), out_dev[1] = any(tree(in...)) (Table 5):
 * 1.0 if every / some element value (in the compute type) is nonzero, else
 * 0.0.  NaN counts as nonzero.  With a relational root this is all(A < x)
 * and any(A < x).  Empty -> all 1.0, any 0.0. */
coot_status coot_all_any(const uint8_t* tree, size_t tree_len, const coot_mat* in, int n_in,
                         double* out_dev, void* ws, size_t ws_bytes, void* stream);

/* out_dev[0] = min, out_dev[1] = max over all elements of tree(in...)
 * (Table 6, both dimensions).  Element values are in the compute type; a
 * NaN anywhere makes both results NaN.  Empty -> COOT_ERR_EMPTY. */
coot_status coot_minmax(const uint8_t* tree, size_t tree_len, const coot_mat* in, int n_in,
                        double* out_dev, void* ws, size_t ws_bytes, void* stream);

/* Several reductions of one tree in ONE pass over the inputs, optionally
 * also storing the element values: `heads` is a mask of COOT_HEAD_* bits;
 * out_dev receives one FP64 per set bit in increasing bit order; `out` (may
 * be NULL) receives the element-wise values as coot_expr_eval would.
 * heads = 0 with out != NULL is coot_expr_eval. */
coot_status coot_expr_reduce(const uint8_t* tree, size_t tree_len, const coot_mat* in, int n_in,
                             unsigned heads, const coot_mat* out, double* out_dev, void* ws,
                             size_t ws_bytes, void* stream);

/* Several trees over the same operands in ONE pass (the delayed evaluation
 * of Section 7 extended to several expressions of one assignment group):
 * every input element is read once for all trees.
 *   trees[k], tree_lens[k]  host buffers, the serialised trees
 *                           (k < n_trees, 1 <= n_trees <= 4); each tree
 *                           reads the first tree_inputs(k) <= n_in operands
 *                           and all trees share tree 0's compute type;
 *   in[0 .. n_in)           the operands (equal shapes, 1 <= n_in <= 4),
 *                           every one read once whether a tree uses it or
 *                           not;
 *   outs                    NULL, or n_trees matrices: tree k is stored
 *                           into outs[k] when outs[k].ptr is not NULL
 *                           (same shape; it may be identical to an input,
 *                           every element's inputs being read before any
 *                           value is stored, and must not overlap another
 *                           stored tree: COOT_ERR_ALIAS);
 *   heads                   NULL, or n_trees masks of COOT_HEAD_* bits;
 *   out_dev                 device FP64 results: tree 0's heads in
 *                           increasing bit order, then tree 1's, ...
 * A tree with neither an output nor heads is an argument error.  Results,
 * summation order and the empty and NaN rules are those of coot_expr_reduce
 * for each tree; the workspace needs room for the partials of every head
 * of every tree. */
coot_status coot_expr_multi(const uint8_t* const* trees, const size_t* tree_lens, int n_trees,
                            const coot_mat* in, int n_in, const coot_mat* outs, const unsigned* heads,
                            double* out_dev, void* ws, size_t ws_bytes, void* stream);

/* coot_expr_multi plus sums along a dimension (Table 6, sum(A, dim)) of any
 * tree in the SAME pass, with no second read of a stored result (the
 * delayed evaluation of Section 7 carried into the sums):
 *   heads[k] may also hold COOT_HEAD_COLSUM and / or COOT_HEAD_ROWSUM;
 *   colsums  NULL, or n_trees matrices: tree k's column sums go to the
 *            1 x n_cols matrix colsums[k] (element j at ptr + j * ld) when
 *            heads[k] has COOT_HEAD_COLSUM;
 *   rowsums  NULL, or n_trees matrices: tree k's row sums go to the
 *            n_rows x 1 matrix rowsums[k] when heads[k] has COOT_HEAD_ROWSUM.
 * Sums are stored in a floating-point type (COOT_ERR_DTYPE otherwise),
 * formed as compensated sums of the compute-type values combined in a fixed
 * order, and rounded once, as coot_sum_dim's; an empty object gives zeros.
 * A sum may not overlap an input, a stored tree or another sum
 * (COOT_ERR_ALIAS).  out_dev holds the full heads as for coot_expr_multi.
 * The workspace holds partial sums and arrival counters; when a shape's
 * partials do not fit in it (more than about 16,000 columns with more than
 * one row segment), the sums are formed by the column / row sum kernels
 * before the pass that stores the trees: same results within rounding,
 * the inputs read again. */
coot_status coot_expr_multi_dims(const uint8_t* const* trees, const size_t* tree_lens, int n_trees,
                                 const coot_mat* in, int n_in, const coot_mat* outs, const unsigned* heads,
                                 double* out_dev, const coot_mat* colsums, const coot_mat* rowsums,
                                 void* ws, size_t ws_bytes, void* stream);

/* Submatrix views (Table 1: .rows(a, b), .cols(c, d), .submat(p, q, r, s),
 * .row(i), .col(j)): the view of rows r0..r1 and columns c0..c1, inclusive,
 * of m, sharing its storage and ld, usable as any input or output.  Bounds
 * outside m -> COOT_ERR_SHAPE.  Host-only. */
coot_status coot_submat(const coot_mat* m, int64_t r0, int64_t c0, int64_t r1, int64_t c1,
                        coot_mat* view);

/* The k-th diagonal of m (Table 1: .diag(k); k > 0 above the main
 * diagonal, k < 0 below) as a 1 x n view with ld = m->ld + 1.  A diagonal
 * outside m -> COOT_ERR_SHAPE.  Host-only. */
coot_status coot_diag(const coot_mat* m, int64_t k, coot_mat* view);

/* Two operands overlap when they share an element: views of one matrix
 * with the same ld are compared by their row and column ranges (so
 * out = A.rows(0, 9) with in = A.rows(10, 19) is allowed); other pairs by
 * the byte ranges they span. */

/* The status word of the kernels' bounded waits on this device, then reset
 * to 0: COOT_OK, or COOT_ERR_TIMEOUT when a wait gave up (the kernel then
 * stopped early; its outputs are incomplete).  Waits on the device
 * (mbarriers of the TMA-staged batched kernel) are bounded at about a
 * second.  Synchronises with the device. */
coot_status coot_device_status(int* status);

/* The device address of pinned host memory (allocated with cudaHostAlloc /
 * cudaMallocHost, or registered with cudaHostRegister), for operands that
 * the kernels read or write in host memory directly: on GB300 the GPU
 * reaches the Grace CPU's memory coherently over NVLink-C2C, so a fused
 * kernel can stream its inputs from host memory and store its outputs
 * there with no staging copy.  `host` may point anywhere inside such an
 * allocation.  Pageable or unknown memory -> COOT_ERR_INVALID_ARG (no
 * pointer is ever guessed); the caller keeps ownership.  Host-only. */
coot_status coot_host_device_pointer(const void* host, void** device);

/* ------------------------------------------------------------------------
 * Statistics along a dimension (Table 6: max/min/sum(A, dim) and the
 * statistics mean/stddev/var(A, dim)), several in ONE pass over the inputs.
 * ---------------------------------------------------------------------- */

#define COOT_STAT_SUM    (1u << 0) /* sum of the line                        */
#define COOT_STAT_MEAN   (1u << 1) /* sum / N                                */
#define COOT_STAT_VAR    (1u << 2) /* sum((v - mean)^2) / (N - 1 + norm_type) */
#define COOT_STAT_STDDEV (1u << 3) /* sqrt(var)                              */
#define COOT_STAT_MIN    (1u << 4) /* smallest element (NaN propagates)      */
#define COOT_STAT_MAX    (1u << 5) /* largest element (NaN propagates)       */
#define COOT_STAT_MASK   0x3Fu

/* Statistics of each line of tree(in...): dim = 0 -> of each column (every
 * out[k] is 1 x n_cols), dim = 1 -> of each row (every out[k] is
 * n_rows x 1).  `stats` is a nonzero mask of COOT_STAT_* bits; `out` is a
 * host array of popcount(stats) device matrices, one per set bit in
 * increasing bit order, all FP32 or all FP64, none overlapping an input or
 * each other.  N is the line length (n_rows for dim 0, n_cols for dim 1).
 * norm_type 0 divides the variance by N - 1 (var of one element is 0),
 * norm_type 1 by N.  N = 0: sums are 0, mean / var / stddev NaN, and
 * min / max COOT_ERR_EMPTY.  Element values and their sums follow the
 * tree's compute type (sums exact per thread, combined as double-word
 * numbers, finished in FP64); a line whose sum of squares leaves the compute
 * type's range gets a NaN variance.  Results do not depend on timing. */
coot_status coot_stats_dim(const uint8_t* tree, size_t tree_len, const coot_mat* in, int n_in,
                           int dim, unsigned stats, int norm_type, const coot_mat* out, void* ws,
                           size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * Batched evaluation: many small matrices of uneven shapes in ONE launch.
 * The paper notes that small matrices leave most of a GPU idle (Section 3)
 * and plans a Cube type for collections of matrices (Section 6); here a
 * persistent kernel walks a work list that covers every matrix, so a batch
 * costs one launch (and can be replayed as one CUDA-graph node).  A work
 * unit is whole columns of one matrix, about 2048 elements.  When two units
 * of every input fit in shared memory, each block stages the next dense
 * unit's inputs with bulk asynchronous copies (TMA, cp.async.bulk) while it
 * computes the current one; its waits are bounded (coot_device_status).
 * ---------------------------------------------------------------------- */

/* One matrix of a batch (device pointers; 8-byte fields).  Every matrix of
 * a batch shares the tree and the storage types given to the call.  Slots
 * the tree does not use may be NULL.  `out` (element-wise values, ld_out)
 * and `colsum` (sum(out, 0): n_cols values, ld_colsum apart) are each
 * optional (NULL). */
typedef struct coot_batch_item {
  const void* in[4];
  int64_t ld_in[4];
  void* out;
  int64_t ld_out;
  void* colsum;
  int64_t ld_colsum;
  int64_t n_rows;
  int64_t n_cols;
} coot_batch_item;

/* Size in bytes of the plan (the items plus the work list) for a batch and
 * the number of work units in it.  Host-only; items is a host array. */
coot_status coot_batch_plan_size(const coot_batch_item* items, int n_items, size_t* bytes,
                                 int64_t* n_work);

/* Validate the items for a tree with n_inputs input slots (every used slot
 * non-NULL, every ld large enough) and write the plan into the HOST buffer
 * plan_host (plan_bytes from coot_batch_plan_size).  The caller copies it
 * to device memory once and passes that copy to coot_expr_eval_batched.
 * Items with n_rows <= 512 are the intended case; any size is accepted. */
coot_status coot_batch_plan_build(const coot_batch_item* items, int n_items, int n_inputs,
                                  void* plan_host, size_t plan_bytes);

/* Evaluate tree over every matrix of the plan in one kernel launch: out =
 * tree(in...) and colsum = sum(out, 0) per matrix.  in_dtypes: host array
 * of n_inputs storage types; out_dtype: storage type of every out;
 * colsum_dtype: COOT_F32 or COOT_F64.  plan_dev: the device copy of a plan
 * built for this batch (the contents are trusted: build it with
 * coot_batch_plan_build), n_items / n_work as built.  Column sums are
 * formed in a fixed order (deterministic). */
coot_status coot_expr_eval_batched(const uint8_t* tree, size_t tree_len, const int32_t* in_dtypes,
                                   int32_t out_dtype, int32_t colsum_dtype, const void* plan_dev,
                                   int n_items, int64_t n_work, void* stream);

/* ------------------------------------------------------------------------
 * Learned launch shapes (not in the paper).  A cost model predicts the
 * log of a kernel's time from features of the call and of a candidate
 * launch shape; with the learned policy on, each call takes the candidate
 * with the lowest prediction.  The model is a 2-layer MLP trained on
 * timings the library measures itself, on the GPU, by the functions below.
 *
 * Parameters: one FP32 array, W1 (d x h, row-major: W1[i * h + j] maps
 * input i to hidden unit j), b1 (h), W2 (h x h), b2 (h), w3 (h), b3 (1);
 * n = d h + h h + 3 h + 1.  Forward: h1 = relu(x W1 + b1), h2 =
 * relu(h1 W2 + b2), y = h2 . w3 + b3.
 * ---------------------------------------------------------------------- */

#define COOT_MODEL_FEATURES 21
#define COOT_MODEL_HIDDEN 64
#define COOT_POLICY_BUILTIN 0
#define COOT_POLICY_LEARNED 1

/* y[b] for the batch x (batch x d, row-major), all device pointers; act
 * receives h1 then h2 (2 * batch * h floats, device) for the gradient. */
coot_status coot_mlp_forward(const float* params, int d, int h, const float* x, int batch, float* y,
                             float* act, void* stream);

/* loss[0] = mean (y - t)^2 and grad = d loss / d params (packed like params)
 * for the batch (x, t) whose forward (y, act) was just computed; work:
 * device scratch of batch * (2 h + 1) floats.  Sums over the batch run in
 * a fixed order: the result is reproducible. */
coot_status coot_mlp_loss_grad(const float* params, int d, int h, const float* x, const float* t,
                               int batch, const float* y, const float* act, float* grad, float* loss,
                               float* work, void* stream);

/* One Adam step (step >= 1 counts the steps for the bias correction):
 * m, v are the caller's zero-initialised moment arrays. */
coot_status coot_mlp_adam(float* params, const float* grad, float* m, float* v, int n, int step,
                          float lr, float beta1, float beta2, float eps, void* stream);

/* The COOT_MODEL_FEATURES features of a call and a candidate launch shape
 * (the model's input; host-only).  kind as coot_set_launch_config (0..3);
 * dtypes: host array of the tree's n_inputs storage types; out_dtype: -1
 * when nothing element-wise is stored; heads: COOT_HEAD_* mask; dense: 1
 * when every operand has ld == n_rows. */
coot_status coot_call_features(const uint8_t* tree, size_t tree_len, int kind, const int32_t* dtypes,
                               int out_dtype, unsigned heads, int64_t n_rows, int64_t n_cols,
                               int dense, int block, int vec, int unroll, int64_t split,
                               float* features);

/* Load cost-model parameters (d = COOT_MODEL_FEATURES, h =
 * COOT_MODEL_HIDDEN; host array of n floats, copied). */
coot_status coot_model_load(const float* params, size_t n);

/* Predicted log time of feature rows (host arrays; host computation,
 * FP64 internally). */
coot_status coot_model_predict(const float* features, int n_rows, float* out);

/* The candidate launch shapes the learned policy chooses among for a kind
 * (0..3): *n receives their count; out (may be NULL) receives up to max of
 * them as {block, vec, unroll, split} int32 quadruples (vec 0: widest
 * aligned; split 0: chosen from the shape).  Host-only. */
coot_status coot_launch_candidates(int kind, int32_t* out, int max, int* n);

/* COOT_POLICY_BUILTIN (default) or COOT_POLICY_LEARNED (needs a loaded
 * model; kinds 0-3).  A launch shape set with coot_set_launch_config still
 * wins over either. */
coot_status coot_set_policy(int policy);

/* ------------------------------------------------------------------------
 * Row sums without a caller workspace.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory where
 * they need the reduction (memory reserved up front by an allocator they do
 * not control, paths that must not synchronise the device the way
 * cudaMalloc / cudaFree can, C callers without a CUDA allocator).  Its
 * scratch is a fixed array of about 4 MiB inside the library's device
 * image, held by every GPU that loads the library until the process exits.
 * ---------------------------------------------------------------------- */

/* Largest row count coot_sum_rows_f32_static accepts (the scratch holds 16
 * FP64 partial sums per row). */
#define COOT_STATIC_MAX_ROWS 32768

/* out = the sum of each row of an FP32 matrix a (n_rows x n_cols, ld),
 * into an FP32 n_rows x 1 out; allocates nothing.  n_rows >
 * COOT_STATIC_MAX_ROWS returns COOT_ERR_UNSUPPORTED; an out that overlaps a
 * returns COOT_ERR_ALIAS.  The first
 * call on a device looks up the scratch's device address
 * (cudaGetSymbolAddress) for that device, with that device current; make
 * that first call before any stream capture.  Each call clears the
 * scratch's counters on `stream` (cudaMemsetAsync) before its kernel.
 * Every call shares the one scratch array: two calls that can run at the
 * same time on the GPU (different streams, or graph branches without an
 * ordering between them) race and give wrong sums. */
coot_status coot_sum_rows_f32_static(const coot_mat* a, const coot_mat* out, void* stream);

/* ------------------------------------------------------------------------
 * Unfused baseline: the paper's own evaluation strategy, one kernel launch
 * per operator node with each intermediate result in an HBM temporary
 * (Section 7: every apply() launches at least one kernel; the last node
 * writes into the destination with its type conversion fused).  Kept to
 * measure what fusion buys on the same GPU.
 * ---------------------------------------------------------------------- */

/* *n_tmp = number of temporaries coot_unfused_eval needs: each holds
 * n_rows * n_cols values of the tree's compute type.  Host-only. */
coot_status coot_unfused_tmp_count(const uint8_t* tree, size_t tree_len, int* n_tmp);

/* out = tree(in...) evaluated node by node.  tmp: device buffer of at least
 * n_tmp * n_rows * n_cols * sizeof(compute type) bytes (caller-owned). */
coot_status coot_unfused_eval(const uint8_t* tree, size_t tree_len, const coot_mat* in, int n_in,
                              const coot_mat* out, void* tmp, size_t tmp_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* COOT_H */
