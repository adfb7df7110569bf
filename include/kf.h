/*
 * kf.h -- C ABI of libkf: fused BLAS-1/BLAS-2 sequences on NVIDIA GB300 (sm_103a).
 *
 * The library follows the kernel-fusion method of Filipovic, Madzin, Fousek
 * and Matyska, "Optimizing CUDA Code By Kernel Fusion -- Application on
 * BLAS": sequences of memory-bound map / reduce / nested map-reduce calls
 * (Section 3.2) are fused so that data shared between calls is read from
 * global memory once.
 *
 * Conventions for every entry point
 *   - Matrices are row major; element (i, j) of an m x n matrix A with
 *     leading dimension lda (elements, lda >= n) is A[i * lda + j].
 *   - "Ap" has length m and "A^T r" length n.  (Algorithm 3 of Section 3.4
 *     indexes p, s by column tiles and q, r by row tiles.)
 *   - All vector/matrix pointers are DEVICE pointers owned by the caller;
 *     the library never allocates, frees or retains them.  16-byte aligned
 *     pointers (and leading dimensions that keep rows 16-byte aligned) take
 *     the vectorised path; others take an element-wise path with the same
 *     results.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls only enqueue work; they do not synchronise, except the
 *     ones documented as synchronous (status/autotune/empirical search).
 *   - `ws` is caller-owned device workspace of at least the size reported by
 *     kf_workspace_size() for the same call and shape.  It must be zero-filled
 *     before its first use (kf_workspace_init does that); every call leaves
 *     its completion counters at zero again, so the same workspace can be
 *     reused for later calls on the same stream.  Calls that share a
 *     workspace must not run concurrently.
 *   - Results are deterministic: cross-block reductions are finished by the
 *     last block to arrive in a fixed order (Section 3.2.2, option (ii)), not
 *     by floating-point atomics.
 *   - Outputs must not alias inputs, except where an entry point says so.
 *   - Sizes may be zero (nothing is read; outputs that are sums over an empty
 *     range are written as the epilogue of zero).
 *   - Every function returns KF_OK (0) or a negative kf_status; on error
 *     nothing has been enqueued and kf_last_error() describes the cause.
 */
#ifndef KF_H
#define KF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int kf_status;
#define KF_OK 0
#define KF_ERR_INVALID_ARG (-1)   /* null pointer, negative size, bad enum   */
#define KF_ERR_SHAPE (-2)         /* inconsistent sizes or leading dims       */
#define KF_ERR_DTYPE (-3)         /* unsupported storage format               */
#define KF_ERR_ALIGN (-4)         /* alignment required by this entry point   */
#define KF_ERR_CYCLE (-5)         /* script dependency cycle                  */
#define KF_ERR_UNDEFINED_VAR (-6) /* script reads a variable never written   */
#define KF_ERR_CUDA (-7)          /* CUDA runtime error (message in last_error) */
#define KF_ERR_NO_MEM (-8)        /* host allocation failed                   */
#define KF_ERR_DEVICE_TIMEOUT (-9) /* a bounded device wait ran out          */
#define KF_ERR_UNSUPPORTED (-10)  /* no kernel instance for this request      */
#define KF_ERR_WORKSPACE (-11)    /* workspace missing or too small           */

/* Storage format of a matrix operand.  The paper is FP32 only (Section 4.1);
 * the row-scaled formats store Q_ij with one FP32 scale s_i per row and
 * represent A_ij ~ s_i * Q_ij. */
typedef enum {
  KF_F32 = 0,
  KF_BF16_ROWSCALE = 1,
  KF_FP8E4M3_ROWSCALE = 2
} kf_dtype;

/* Call kinds whose workspace needs differ (kf_workspace_size). */
typedef enum {
  KF_SEQ_BICGK = 0,
  KF_SEQ_GEMVER = 1,
  KF_SEQ_GESUMMV = 2,
  KF_SEQ_ATAX = 3,
  KF_SEQ_AXPYDOT = 4,
  KF_SEQ_WAXPBY = 5,
  KF_SEQ_GEMV = 6,
  KF_SEQ_GEMVT = 7,
  KF_SEQ_DOT = 8,
  KF_SEQ_SGEMVT = 9
} kf_seq;

/* Library version string (static storage). */
const char* kf_version(void);

/* Message of the last error on the calling thread (valid until the next
 * libkf call on that thread). */
const char* kf_last_error(void);

/* Number of SMs of the current device (152 on GB300). */
kf_status kf_device_sm_count(int* sm_count);

/* Bytes of workspace needed by call kind `seq` on an m x n problem (vectors:
 * m = 1, n = length) for every tuning the library may pick. */
kf_status kf_workspace_size(kf_seq seq, int64_t m, int64_t n, kf_dtype fmt, size_t* bytes);

/* Zero `bytes` of workspace on `stream` (required once before first use). */
kf_status kf_workspace_init(void* ws, size_t bytes, void* stream);

/* Synchronise `stream` and read the device error word at the start of `ws`:
 * returns KF_ERR_DEVICE_TIMEOUT (and clears the word) if a bounded wait of
 * an earlier call on this workspace ran out, KF_OK otherwise. */
kf_status kf_workspace_status(void* ws, void* stream);

/* Bound of every kernel wait on data (not in the paper: its kernels wait on
 * nothing but kernel boundaries).  The staged matrix pass and ATAX wait for
 * bulk asynchronous copies on mbarriers; each such wait gives up after
 * limit_ns (default 1 s), after which the block records the timeout in the
 * workspace's error word (kf_workspace_status reports KF_ERR_DEVICE_TIMEOUT),
 * lets the copies already in flight land within the default bound, and
 * returns, so the context stays usable.  Process-wide; applies to launches
 * enqueued after the call.  Range KF_WAIT_LIMIT_MIN_NS..KF_WAIT_LIMIT_MAX_NS,
 * else KF_ERR_INVALID_ARG.  A limit shorter than a copy's latency makes
 * waits run out on healthy copies (wrong results, reported by the status). */
#define KF_WAIT_LIMIT_MIN_NS ((uint64_t)1000)
#define KF_WAIT_LIMIT_MAX_NS ((uint64_t)60000000000ull)
kf_status kf_set_wait_limit_ns(uint64_t limit_ns);
kf_status kf_get_wait_limit_ns(uint64_t* limit_ns);

/* Probe of the timeout path shared by every bounded wait (a diagnostic, not
 * in the paper): one thread of one block waits, bounded by limit_ns, on an
 * mbarrier phase that nothing completes, so the wait runs out; the kernel
 * then sets the error word at the start of `ws` (>= 256 bytes) and returns.
 * kf_workspace_status(ws) afterwards reports KF_ERR_DEVICE_TIMEOUT.
 * waited_ns (device pointer or NULL) receives the nanoseconds the wait took
 * by the global timer.  Enqueued on `stream`; no fault, trap or unbounded
 * wait is involved. */
kf_status kf_wait_probe(uint64_t limit_ns, void* ws, size_t ws_bytes, unsigned long long* waited_ns,
                        void* stream);

/* ------------------------------------------------------------------------
 * Fused sequences (Table 1 of Section 4.1).  Each is one pass of the fused
 * kernels the planner emits for the canonical script of the sequence.
 * ---------------------------------------------------------------------- */

/* BiCGK (Section 3.4, Listing 1, Algorithm 3): q = A p and s = A^T r with a
 * single read of A.  A: m x n (fmt KF_F32, or row-scaled Q with row_scale of
 * length m); p, s: length n; q, r: length m.  One kernel launch. */
kf_status kf_bicgk(int64_t m, int64_t n, const void* A, int64_t lda, kf_dtype fmt,
                   const float* row_scale, const float* p, const float* r, float* q, float* s,
                   void* ws, size_t ws_bytes, void* stream);

/* GEMVER (Table 1): B = A + u1 v1^T + u2 v2^T; x = beta B^T y + z;
 * w = alpha B x.  A, B: n x n (B written, ldb >= n); all vectors length n.
 * w needs all of x (a global barrier, Section 3.2.2).  Two forms: two
 * launches, the second rereading B from the rows the first wrote last; or
 * kf_gemver_single's one cooperative launch.  kf_gemver takes the single
 * launch where its tuning on first use measured it more than 2 % faster at
 * that size class (tuning cache key "gemver_form log2(n)"), else two
 * launches. */
kf_status kf_gemver(int64_t n, const float* A, int64_t lda, const float* u1, const float* v1,
                    const float* u2, const float* v2, const float* y, const float* z, float alpha,
                    float beta, float* B, int64_t ldb, float* x, float* w, void* ws,
                    size_t ws_bytes, void* stream);

/* GEMVER in one cooperative launch (Table 1; Section 4.2's persistent-thread
 * remark): the same results as kf_gemver (B bit for bit; x and w in another
 * fixed summation order), with the global barrier on x crossed by bounded
 * grid-wide barriers instead of a kernel boundary, the cross-block sums of x
 * and w finished by the whole grid, and B read back in reverse row order.
 * Needs n a multiple of 4 (n >= 8), 16-byte aligned operands, lda and ldb
 * multiples of 4 and B not in place of A (else KF_ERR_UNSUPPORTED).  ws:
 * kf_workspace_size(KF_SEQ_GEMVER, n, n).  kf_gemver picks this form when
 * its tuning on first use measured it faster at that size class. */
kf_status kf_gemver_single(int64_t n, const float* A, int64_t lda, const float* u1, const float* v1,
                           const float* u2, const float* v2, const float* y, const float* z, float alpha,
                           float beta, float* B, int64_t ldb, float* x, float* w, void* ws, size_t ws_bytes,
                           void* stream);

/* GEMVER with row-scaled low-precision storage (not in the paper, whose
 * kernels are FP32 only).  A is given as codes QA (fmt BF16 or FP8-E4M3,
 * row stride lda elements) with per-row scales sA (kf_quantize_rows):
 * Ahat_ij = sA_i QA_ij.  B = Ahat + u1 v1^T + u2 v2^T is stored in the same
 * format, codes QB (row stride ldb, must not alias QA) and scales sB, by
 * this rule (FP32 arithmetic, in this order; QMAX = 1 for BF16, 448 for
 * E4M3):
 *   sB_i  = (sA_i * QMAX + |u1_i| max_j |v1_j| + |u2_i| max_j |v2_j|) / QMAX
 *           (1 when that is 0): a per-row bound on |B_ij|, so no code
 *           saturates and no second pass over B is needed for its amax;
 *   b_ij  = fma(u2_i, v2_j, fma(u1_i, v1_j, sA_i * QA_ij));
 *   QB_ij = round-to-nearest-even of b_ij * (1 / sB_i) into the format
 *           (E4M3 saturating).
 * Then x = beta Bhat^T y + z and w = alpha Bhat x with Bhat_ij = sB_i QB_ij,
 * the stored matrix, accumulated in FP32.  Launches: a norm pre-pass and
 * the two matrix passes of kf_gemver.  ws: kf_workspace_size(KF_SEQ_GEMVER,
 * n, n, fmt).  Errors: KF_ERR_DTYPE (fmt KF_F32), KF_ERR_SHAPE, KF_ERR_INVALID_ARG,
 * KF_ERR_WORKSPACE. */
kf_status kf_gemver_q(int64_t n, const void* QA, int64_t lda, kf_dtype fmt, const float* sA, const float* u1,
                      const float* v1, const float* u2, const float* v2, const float* y, const float* z,
                      float alpha, float beta, void* QB, int64_t ldb, float* sB, float* x, float* w, void* ws,
                      size_t ws_bytes, void* stream);

/* SGEMVT (Table 1): x = beta A^T y + z; w = alpha A x.  A: m x n; y, w:
 * length m; z, x: length n.  w needs all of x (a global barrier, Section
 * 3.2.2).  Two forms, each reading A twice: two launches, the second
 * walking each row group from the rows the first read last (then still in
 * L2); or kf_sgemvt_single's one cooperative launch.  kf_sgemvt takes the
 * single launch where its tuning on first use measured it more than 2 %
 * faster at that size class (tuning cache key "sgemvt_form log2(m)
 * log2(n)"), else two launches.  ws: kf_workspace_size(KF_SEQ_SGEMVT, m, n).
 * Errors: KF_ERR_INVALID_ARG, KF_ERR_SHAPE, KF_ERR_WORKSPACE. */
kf_status kf_sgemvt(int64_t m, int64_t n, const float* A, int64_t lda, const float* y, const float* z,
                    float alpha, float beta, float* x, float* w, void* ws, size_t ws_bytes, void* stream);

/* SGEMVT in one cooperative launch: the kernel of kf_gemver_single without
 * the rank-one updates and the stored matrix; the second phase rereads A in
 * reverse row order.  x and w are sums in another fixed order than the two
 * launches'.  Needs m >= 8, n a multiple of 4, lda a multiple of 4 and
 * 16-byte aligned operands (else KF_ERR_UNSUPPORTED).  ws:
 * kf_workspace_size(KF_SEQ_SGEMVT, m, n). */
kf_status kf_sgemvt_single(int64_t m, int64_t n, const float* A, int64_t lda, const float* y, const float* z,
                           float alpha, float beta, float* x, float* w, void* ws, size_t ws_bytes, void* stream);

/* GESUMMV (Table 1): y = alpha A x + beta B x.  A, B: m x n with the same
 * leading dimension; x: length n; y: length m.  One launch; x is read once
 * per column strip for both matrices. */
kf_status kf_gesummv(int64_t m, int64_t n, const float* A, const float* B, int64_t lda,
                     const float* x, float alpha, float beta, float* y, void* ws, size_t ws_bytes,
                     void* stream);

/* ATAX (Table 1): y = A^T (A x).  A: m x n; x, y: length n.  One read of A
 * by blocks that own whole rows (rows staged by bulk asynchronous copies),
 * plus a small finishing launch; falls back to two passes (t = A x, then
 * y = A^T t, the paper's form) when rows are not 16-byte aligned or n > 16384.
 * Device waits are bounded: see kf_workspace_status. */
kf_status kf_atax(int64_t m, int64_t n, const float* A, int64_t lda, const float* x, float* y,
                  void* ws, size_t ws_bytes, void* stream);

/* AXPYDOT (Table 1): z = w - alpha v; r = z^T u.  Vectors length n; r is one
 * device float.  One launch.  The cross-block sum of r is done in double for
 * n >= 2^26. */
kf_status kf_axpydot(int64_t n, const float* w, const float* v, const float* u, float alpha,
                     float* z, float* r, void* ws, size_t ws_bytes, void* stream);

/* WAXPBY (Table 1): w = alpha x + beta y.  One launch, no workspace. */
kf_status kf_waxpby(int64_t n, float alpha, const float* x, float beta, const float* y, float* w,
                    void* stream);

/* ------------------------------------------------------------------------
 * Elementary functions (Section 3.3): one kernel each, out of place unless
 * stated.  They form the unfused per-call chains.
 * ---------------------------------------------------------------------- */

/* y = alpha A x + beta y0 (y0 may be NULL when beta == 0).  A: m x n. */
kf_status kf_gemv(int64_t m, int64_t n, const void* A, int64_t lda, kf_dtype fmt,
                  const float* row_scale, float alpha, const float* x, float beta,
                  const float* y0, float* y, void* ws, size_t ws_bytes, void* stream);

/* x = alpha A^T y + beta x0 (x0 may be NULL when beta == 0).  A: m x n. */
kf_status kf_gemvt(int64_t m, int64_t n, const void* A, int64_t lda, kf_dtype fmt,
                   const float* row_scale, float alpha, const float* y, float beta,
                   const float* x0, float* x, void* ws, size_t ws_bytes, void* stream);

/* B = A + alpha u v^T.  u: length m, v: length n.  B may equal A (in place,
 * then ldb must equal lda). */
kf_status kf_ger(int64_t m, int64_t n, const float* A, int64_t lda, float alpha, const float* u,
                 const float* v, float* B, int64_t ldb, void* stream);

/* out = alpha x + beta y (AXPY when out == y and beta == 1; in place allowed). */
kf_status kf_axpby(int64_t n, float alpha, const float* x, float beta, const float* y, float* out,
                   void* stream);

/* out = alpha x (SCAL; in place allowed). */
kf_status kf_scal(int64_t n, float alpha, const float* x, float* out, void* stream);

/* out = w + y + z (VADD of Table 1; in place allowed). */
kf_status kf_vadd3(int64_t n, const float* w, const float* y, const float* z, float* out,
                   void* stream);

/* C = A + B (MADD of Table 1).  m x n matrices with leading dimensions
 * lda, ldb, ldc >= n; C may be A or B (in place).  Contiguous operands take
 * one vector pass over m n elements.  Errors: KF_ERR_INVALID_ARG (null
 * operand), KF_ERR_SHAPE (leading dimension below n). */
kf_status kf_madd(int64_t m, int64_t n, const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                  int64_t ldc, void* stream);

/* *out = x . y (one device float). */
kf_status kf_dot(int64_t n, const float* x, const float* y, float* out, void* ws, size_t ws_bytes,
                 void* stream);

/* ------------------------------------------------------------------------
 * Row-scaled low-precision storage (not in the paper, which is FP32 only).
 * ---------------------------------------------------------------------- */

/* Quantise an FP32 matrix row by row: s_i = amax_i / QMAX (QMAX = 1 for
 * BF16, 448 for E4M3; s_i = 1 for an all-zero row), Q_ij = round-to-nearest-
 * even of (A_ij / s_i) in the format, saturating at +-448 for E4M3.  Q is
 * written densely (leading dimension n), 2 bytes per element for BF16, 1 for
 * E4M3; row_scale gets m floats. */
kf_status kf_quantize_rows(int64_t m, int64_t n, const float* A, int64_t lda, kf_dtype fmt, void* Q,
                           float* row_scale, void* stream);

/* ------------------------------------------------------------------------
 * Tuning (Section 3.2: block size and serial iterations are part of a
 * fusion implementation).  A tuning applies to matrix passes launched
 * afterwards in the calling process.  warps in {4, 8}; vec (16-byte chunks
 * per lane per row) in {1, 2, 4}; unroll (rows per batch) in {1, 2, 4, 8};
 * groups = row groups per column strip (0 = fill one wave of resident
 * blocks); stages = depth of each warp's bulk-copy ring (1..8), or 0 for
 * direct 16-byte loads.  warps = 0 restores the automatic choice (the
 * default).  A combination without a compiled instance falls back to the
 * default instance of the same op shape.
 * ---------------------------------------------------------------------- */
kf_status kf_set_matrix_tuning(int warps, int vec, int unroll, int groups, int stages);
kf_status kf_get_matrix_tuning(int* warps, int* vec, int* unroll, int* groups, int* stages);

/* ------------------------------------------------------------------------
 * Scripts and plans (Sections 3.1-3.2: the script of elementary calls, the
 * data-dependency graph, fusions, their combination and its prediction).
 *
 * A script declares variables (vectors of length n, row-major m x n
 * matrices with leading dimension n, device float scalars), marks inputs
 * and outputs, and lists calls in order.  Every variable, inputs, outputs
 * and temporaries alike, is bound to caller-owned device memory at
 * execution (bindings[var_id]); a fused plan may leave temporaries that
 * stay on chip unwritten.  Call semantics (BLAS conventions):
 *   AXPBY  out = a x + b y          ins (x, y)        scalars (a, b)   [AXPY: out = y, b = 1]
 *   SCAL   out = a x                ins (x)           scalars (a)
 *   DOT    out = x . y  (scalar)    ins (x, y)
 *   VADD   out = w + y + z          ins (w, y, z)
 *   GEMV   out = a A x + b y0       ins (A, x[, y0])  scalars (a, b)   out may not be x
 *   GEMVT  out = a A^T y + b x0     ins (A, y[, x0])  scalars (a, b)   out may not be y
 *   GER    out = A + a u v^T        ins (A, u, v)     scalars (a)      out may be A (in place)
 * Missing scalars default to a = 1 and b = 1 (AXPBY) / b = 1 when y0 or x0
 * is given, else 0.
 *
 * Fusion rules (Section 3.2): calls of one fusion have the same nesting
 * depth and iteration space (vectors of one length, or matrices of one
 * shape); no call consumes a reduction result (DOT, GEMV, GEMVT) of the
 * same fusion, except linear maps (AXPBY, SCAL, VADD) of row or column
 * results, which run after the last-block barrier; a fusion is convex in
 * the dependency graph; at most 4 matrix ops over at most 2 matrices and 2
 * GEMV results per matrix pass; at most 6 input vectors, 4 outputs and 4
 * dots per vector pass.  Plans are enumerated call by call in script order
 * (at most max_plans).
 * ---------------------------------------------------------------------- */
typedef struct kf_script kf_script;
typedef struct kf_plan kf_plan;

typedef enum {
  KF_OP_AXPBY = 0,
  KF_OP_SCAL = 1,
  KF_OP_DOT = 2,
  KF_OP_VADD = 3,
  KF_OP_GEMV = 4,
  KF_OP_GEMVT = 5,
  KF_OP_GER = 6
} kf_op;

typedef enum {
  KF_PLAN_UNFUSED = 0,   /* one kernel per call                                   */
  KF_PLAN_GREEDY = 1,    /* fewest kernels                                        */
  KF_PLAN_ANALYTIC = 2,  /* least predicted time (kf_plan_predicted_us)           */
  KF_PLAN_INDEX = 3      /* the index-th plan of the enumeration                  */
} kf_plan_mode;

typedef struct {
  int mode;       /* kf_plan_mode                         */
  int max_plans;  /* enumeration cap (<= 0: 20000)        */
  int index;      /* KF_PLAN_INDEX                        */
} kf_plan_options;

kf_status kf_script_create(kf_script** out);
void kf_script_destroy(kf_script* s);
kf_status kf_script_vector(kf_script* s, const char* name, int64_t n, int* var_id);
kf_status kf_script_matrix(kf_script* s, const char* name, int64_t m, int64_t n, int* var_id);
/* A matrix whose rows are ld elements apart (ld >= n, else KF_ERR_SHAPE):
 * an m x n view of a wider row-major FP32 array, bound to the pointer of its
 * first element.  kf_script_matrix is the case ld = n.  Every kernel the
 * planner emits takes the stride (matrix passes, single-pass ATAX); rows not
 * 16 bytes apart take the element-wise load path. */
kf_status kf_script_matrix_ld(kf_script* s, const char* name, int64_t m, int64_t n, int64_t ld, int* var_id);
kf_status kf_script_scalar(kf_script* s, const char* name, int* var_id);
kf_status kf_script_input(kf_script* s, int var_id);
kf_status kf_script_output(kf_script* s, int var_id);
kf_status kf_script_call(kf_script* s, kf_op op, const int* outs, int n_out, const int* ins, int n_in,
                         const double* scalars, int n_scalars);
/* Check shapes and that every read variable is an input or written earlier
 * (KF_ERR_SHAPE / KF_ERR_UNDEFINED_VAR). */
kf_status kf_script_validate(const kf_script* s);
/* Number of legal plans (at most cap); *truncated = 1 when the cap was hit. */
kf_status kf_plan_count(const kf_script* s, int cap, int* count, int* truncated);
kf_status kf_plan_build(const kf_script* s, const kf_plan_options* opt, kf_plan** out);
void kf_plan_destroy(kf_plan* p);
kf_status kf_plan_workspace_size(const kf_plan* p, size_t* bytes);
kf_status kf_plan_kernel_count(const kf_plan* p, int* n);
/* Analytic prediction (microseconds), the paper's predictor (Section 3.2:
 * transfer and compute times summed separately, max(t_t, t_c)) plus a fixed
 * cost per kernel: sum over kernels of max(bytes moved / model bandwidth,
 * flops / FP32 rate) + launch cost (bandwidth and launch cost set by
 * kf_planner_set_model). */
kf_status kf_plan_predicted_us(const kf_plan* p, double* us);
kf_status kf_planner_set_model(double bw_gbs, double launch_us);
/* Features of a plan for the learned cost model (16 floats). */
kf_status kf_plan_features(const kf_script* s, const kf_plan* p, float* out, int cap, int* n);
/* For every enumerated plan (at most cap, in KF_PLAN_INDEX order): its 16
 * features (feats: cap x 16), analytic prediction and kernel count (any
 * output may be NULL). */
kf_status kf_plan_enumerate_info(const kf_script* s, int cap, float* feats, double* pred_us, int* kernels,
                                 int* count);
/* JSON: kernels, their calls (script order) and bytes, prediction.  A matrix
 * kernel also gives "order", its calls in the order the kernel runs them,
 * and "specialised", whether a specialised instance exists for that order.
 * The planner's call-order search (Section 3.2, variant (i)) picks the order:
 * the first legal one, script order first, whose op signature has a
 * compiled specialised instance.  Calls that share a variable, one of them
 * writing it, keep script order (a GER writes the matrix it updates), so
 * every admissible order gives the same results bit for bit. */
kf_status kf_plan_describe(const kf_plan* p, char* buf, size_t cap, size_t* needed);
/* Enqueue the plan's kernels on `stream`.  bindings[var_id] is the device
 * address of each script variable (one device float for a scalar); ws holds
 * at least kf_plan_workspace_size bytes.  Every kernel's bindings and
 * workspace are checked before the first launch: on KF_ERR_INVALID_ARG (a
 * variable not bound) or KF_ERR_WORKSPACE nothing has been enqueued. */
kf_status kf_plan_execute(const kf_plan* p, void* const* bindings, int n_bindings, void* ws, size_t ws_bytes,
                          void* stream);
/* Synchronous: run once, then time `reps` executions with CUDA events on
 * `stream`; the median in milliseconds (empirical search, Section 3.2). */
kf_status kf_plan_time(const kf_plan* p, void* const* bindings, int n_bindings, void* ws, size_t ws_bytes,
                       void* stream, int reps, float* median_ms);

/* ------------------------------------------------------------------------
 * Plan selection.  The paper ranks the implementations of a script with an
 * additive predictor and can search them empirically (Section 3.2).
 * kf_plan_select picks one of the enumerated plans (at most max_plans;
 * <= 0: 2000):
 *   KF_SELECT_ANALYTIC    least analytic prediction; no GPU work, ws and
 *                         bindings unused;
 *   KF_SELECT_MLP         the learned cost model (kf_mlp_*, 16 inputs, 64
 *                         hidden units) scores every plan on the GPU from its
 *                         features standardised as (f - mean) * inv_std (the
 *                         score estimates ln(ms), see kf_cost_model); the
 *                         lowest score ranks first; with top_k <= 1 the first-ranked
 *                         plan is kept untimed, else the top_k best-ranked
 *                         plans are timed on the bound data and the fastest
 *                         kept (top_k >= the plan count: every plan is timed,
 *                         the exhaustive fallback);
 *   KF_SELECT_EXHAUSTIVE  every plan is timed; the fastest is kept.
 * Timing is kf_plan_time's (one warm-up run, median of `reps` >= 1; <= 0:
 * 3) and writes the plans' outputs and in-place operands.  ws: at least
 * kf_plan_select_workspace_size bytes, zero-filled before its first use
 * (the plans' region, then the model's inputs and outputs).  Synchronous on
 * `stream`.  *out is a new plan (kf_plan_destroy); info may be NULL.
 * Errors: KF_ERR_INVALID_ARG (no model for KF_SELECT_MLP, missing bindings
 * when timing), KF_ERR_WORKSPACE, KF_ERR_UNSUPPORTED (no legal plan).
 * ---------------------------------------------------------------------- */
typedef enum { KF_SELECT_ANALYTIC = 0, KF_SELECT_MLP = 1, KF_SELECT_EXHAUSTIVE = 2 } kf_select_mode;

typedef struct {
  int mode;       /* kf_select_mode                          */
  int max_plans;  /* enumeration cap (<= 0: 2000)            */
  int top_k;      /* KF_SELECT_MLP: best-ranked plans timed  */
  int reps;       /* timed runs per plan (<= 0: 3)           */
  float margin;   /* KF_SELECT_MLP: also time every plan whose score is
                     within `margin` of the best score (ln(ms) units; at
                     most 64 plans in all); 0: top_k only             */
} kf_select_options;

typedef struct {
  const float* params;   /* device: kf_mlp_param_count(16, 64) floats   */
  float mean[16];        /* host: feature standardisation               */
  float inv_std[16];
  float analytic_weight; /* score = MLP output + analytic_weight *
                            ln(analytic prediction in ms); 1: the network
                            learned the residual of the analytic model   */
} kf_cost_model;

typedef struct {
  int index;        /* chosen plan, in KF_PLAN_INDEX order                 */
  int count;        /* plans enumerated                                    */
  int timed;        /* plans timed                                         */
  float best_ms;    /* median of the chosen plan (0 when nothing was timed) */
  double predicted; /* MLP: the chosen plan's score; otherwise analytic us */
} kf_select_info;

kf_status kf_plan_select_workspace_size(const kf_script* s, int max_plans, size_t* bytes);
kf_status kf_plan_select(const kf_script* s, const kf_select_options* opt, const kf_cost_model* model,
                         void* const* bindings, int n_bindings, void* ws, size_t ws_bytes, void* stream, kf_plan** out,
                         kf_select_info* info);
/* Median time (ms) of every enumerated plan, in KF_PLAN_INDEX order (ms:
 * room for max_plans floats): the data of the exhaustive search, which
 * scores the cost models.  Workspace and timing as kf_plan_select. */
kf_status kf_plan_time_all(const kf_script* s, int max_plans, void* const* bindings, int n_bindings, void* ws,
                           size_t ws_bytes, void* stream, int reps, float* ms, int* count);

/* ------------------------------------------------------------------------
 * Training the learned cost model (not in the paper, whose predictor is the
 * additive one of Section 3.2) on plan timings the caller measured with
 * kf_plan_time / kf_plan_time_all, features from kf_plan_enumerate_info.
 * Everything runs in the library: the features are standardised as
 * (f - mean) / (std + 1e-6) (population std, double); the target of sample i
 * is ln(measured_ms[i]) - analytic_weight * ln(max(analytic_us[i], 1e-3) *
 * 1e-3), minus the mean target of its script when centre_per_script is set
 * (script_ids required: only differences between one script's plans decide
 * a choice); the network (kf_mlp_*, KF_PLAN_NFEATURES -> 64 -> 64 -> 1)
 * starts from params_init (device, may be NULL) or from He-uniform weights
 * u * sqrt(6 / fan_in) with zero biases, u the SplitMix64 stream of `seed`
 * (counter-based, stream id 15) at the parameter's index; then `epochs`
 * full-batch Adam steps (kf_mlp_loss_grad, kf_mlp_adam).
 *   features     host, count x KF_PLAN_NFEATURES, row major
 *   measured_ms  host, count (> 0);  analytic_us: host, count
 *   script_ids   host, count, or NULL
 *   params       device output, kf_mlp_param_count(16, 64) floats
 *   ws           device, kf_planner_train_workspace_size bytes
 *   model        output: params = `params`, the standardisation and
 *                analytic_weight, ready for kf_plan_select
 *   loss_out     host, loss_cap floats (may be NULL with loss_cap 0): the
 *                mean squared error before step 1, every loss_every steps,
 *                and after the last step; *n_loss (may be NULL) the count.
 * Synchronous on `stream`.  Errors: KF_ERR_INVALID_ARG (sizes, options, a
 * non-positive time), KF_ERR_WORKSPACE, KF_ERR_CUDA.
 * ---------------------------------------------------------------------- */
#define KF_PLAN_NFEATURES 16

typedef struct {
  int epochs;             /* full-batch Adam steps (>= 1)                      */
  float lr;               /* Adam step size                                   */
  float beta1, beta2, eps;
  float analytic_weight;  /* weight of ln(analytic ms) in the target and score */
  int centre_per_script;  /* centre the targets per script (needs script_ids) */
  int loss_every;         /* record the loss every this many steps (0: no)   */
  uint64_t seed;          /* initial weights when params_init is NULL         */
} kf_train_options;

kf_status kf_planner_train_workspace_size(int count, int d_in, size_t* bytes);
kf_status kf_planner_train(const float* features, const double* measured_ms, const double* analytic_us,
                           const int64_t* script_ids, int count, int d_in, const kf_train_options* opt,
                           const float* params_init, float* params, void* ws, size_t ws_bytes, void* stream,
                           kf_cost_model* model, float* loss_out, int loss_cap, int* n_loss);

/* ------------------------------------------------------------------------
 * Autotuning (Section 3.2: block size and serial iterations are part of a
 * fusion implementation; routines are benchmarked once per architecture).
 * kf_autotune_plan runs, for every kernel of the plan on the bound data,
 * each compiled implementation that fits its op shape (warps, 16-byte chunks
 * per lane, rows per batch, direct loads or a bulk-copy ring of depth 2..4,
 * and for matrices of at most 16384 rows also 16, 32 or 64 row groups in
 * place of one wave's worth; for vector passes rows in flight and grid
 * size), each timed as the mean
 * of `reps` back-to-back launches (best of two rounds, after a warm-up of
 * the current choice), and stores the fastest in a process-wide tuning
 * cache (keeping the current choice unless the fastest gains more than 2 %,
 * since short timings are noisy), keyed by op signature, storage
 * format and size class (powers of two of m and n).  Automatic launches
 * (every entry point, unless kf_set_matrix_tuning fixed a tuning) consult
 * the cache.  Synchronous; it writes the plan's outputs and in-place
 * operands.  *tuned_ms / *auto_ms: sum over kernels of the best time and
 * of the time with the tuning the cache had before.  The cache can be
 * saved and loaded (text, keyed by device name and SM count; entries for
 * another device are ignored).
 * ---------------------------------------------------------------------- */
kf_status kf_autotune_plan(const kf_plan* p, void* const* bindings, int n_bindings, void* ws, size_t ws_bytes,
                           void* stream, int reps, float* tuned_ms, float* auto_ms);
/* Tuning on first use.  reps > 0: every automatic matrix- or vector-pass
 * launch (any entry point, no tuning fixed by kf_set_matrix_tuning) whose
 * tuning-cache key has no entry first runs the empirical search of
 * kf_autotune_plan on its own operands, `reps` timed runs per candidate,
 * synchronously, and stores the winner; later launches of the key take it
 * from the cache.  The search runs the call's kernel repeatedly, so calls
 * that update an operand in place (GER into its own input, in-place GEMVER)
 * must not make a first launch of a key while it is enabled.  No search
 * runs while the stream is being captured.  reps = 0 (the default) turns
 * it off; reps > 100 is KF_ERR_INVALID_ARG. */
kf_status kf_set_autotune(int reps);
kf_status kf_get_autotune(int* reps);
kf_status kf_tune_cache_clear(void);
kf_status kf_tune_cache_entries(int* n);
kf_status kf_tune_cache_save(const char* path);
kf_status kf_tune_cache_load(const char* path, int* loaded);

/* ------------------------------------------------------------------------
 * Batched BiCGK / GESUMMV: many independent instances of uneven sizes in one
 * persistent launch (not in the paper; its persistent-thread remark is in
 * Section 4.2).  Each instance is described by device pointers:
 *   BiCGK   : y = A x (q = A p), s = A^T r        (B unused, alpha/beta unused)
 *   GESUMMV : y = alpha A x + beta B x             (r, s unused)
 * with A (and B) m x n, leading dimension lda >= n (any alignment).  The
 * host tables (descriptors, tiles sorted largest first) live in the batch
 * object; kf_batched_upload copies them into the caller's workspace
 * (synchronous), after which kf_batched_launch may be enqueued or captured
 * any number of times: its work queue and per-instance counters reset
 * themselves.  band_rows (a multiple of 32; 0 = 128) is the tile height.
 * Each instance's result equals the same instance batched alone (fixed
 * reduction order per instance).
 * ---------------------------------------------------------------------- */
typedef struct {
  int64_t m, n, lda;
  const float* A;
  const float* B;
  const float* x;
  const float* r;
  float* y;
  float* s;
  float alpha, beta;
} kf_batch_desc;

typedef struct kf_batched kf_batched;

kf_status kf_batched_create(kf_seq seq, const kf_batch_desc* descs, int count, int band_rows, kf_batched** out);
void kf_batched_destroy(kf_batched* b);
kf_status kf_batched_workspace_size(const kf_batched* b, size_t* bytes);
/* Tiles of one launch and its algorithmic bytes (matrices once, vectors once). */
kf_status kf_batched_info(const kf_batched* b, int* ntiles, double* bytes);
kf_status kf_batched_upload(const kf_batched* b, void* ws, size_t ws_bytes, void* stream);
kf_status kf_batched_launch(const kf_batched* b, void* ws, size_t ws_bytes, void* stream);
/* Autotuned tile height: each candidate band height (32..512 rows) is
 * uploaded into `ws` and timed `reps` times (synchronous); the workspace
 * must hold the largest candidate (kf_batched_workspace_bound). */
kf_status kf_batched_workspace_bound(kf_seq seq, const kf_batch_desc* descs, int count, size_t* bytes);
kf_status kf_batched_autotune(kf_seq seq, const kf_batch_desc* descs, int count, void* ws, size_t ws_bytes,
                              void* stream, int reps, int* best_band_rows, float* best_ms);
/* Capture one launch into a CUDA graph (cudaGraphExec_t returned as void*). */
kf_status kf_batched_graph_create(const kf_batched* b, void* ws, size_t ws_bytes, void** graph_exec);
kf_status kf_batched_graph_launch(void* graph_exec, void* stream);
void kf_batched_graph_destroy(void* graph_exec);

/* ------------------------------------------------------------------------
 * Learned cost model (not in the paper, whose predictor is the additive
 * one of Section 3.2): a 3-layer perceptron with ReLU activations
 *   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), f = W3 h2 + b3,
 * 64 hidden units, d_in <= 32 inputs, trained with the mean squared error
 * on log plan time and Adam (Kingma and Ba 2015, Algorithm 1).  Parameters
 * are one caller-owned device FP32 array: W1 (64 x d_in, row major), b1
 * (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1).  X is batch x d_in row
 * major.  Gradients are summed over blocks in a fixed order.
 * ---------------------------------------------------------------------- */
kf_status kf_mlp_param_count(int d_in, int hidden, int* count);
kf_status kf_mlp_workspace_size(int d_in, int hidden, int batch, size_t* bytes);
kf_status kf_mlp_forward(const float* params, int d_in, int hidden, const float* X, int batch, float* out,
                         void* stream);
/* *loss (device float, may be NULL) = mean (f - y)^2; grad = dL/dparams. */
kf_status kf_mlp_loss_grad(const float* params, int d_in, int hidden, const float* X, const float* y, int batch,
                           float* grad, float* loss, void* ws, size_t ws_bytes, void* stream);
/* One Adam step (step counts from 1) on params with moments m, v. */
kf_status kf_mlp_adam(float* params, const float* grad, float* m, float* v, int count, int step, float lr, float b1,
                      float b2, float eps, void* stream);

/* ------------------------------------------------------------------------
 * BiCGK for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a library convenience.
 *
 * Some callers cannot call cudaMalloc or any allocating routine where they
 * need BiCGK (a framework that forbids allocation while it records work, a
 * host whose device memory belongs to another allocator, a C program with
 * no device allocator).  kf_bicgk_noalloc computes what kf_bicgk computes
 * for FP32 A (q = A p, s = A^T r, one read of A) but takes no
 * workspace: its scratch is a fixed array of KF_BICGK_NOALLOC_SCRATCH_BYTES
 * in the library's device image, present on every GPU that loads the
 * library until the process exits.  It allocates nothing.
 *   - Shapes whose scratch would exceed the array (about m, n <= 8192 when
 *     m = n) return KF_ERR_SHAPE; use kf_bicgk with a workspace for those.
 *   - The first call on a device, with that device current, looks up the
 *     array's device address and caches it; make that first call before any
 *     stream capture.
 *   - Each call clears the array's counters on `stream` before its launch.
 *   - The kernel shape is the one kf_bicgk takes without a search (a tuning
 *     fixed by kf_set_matrix_tuning, else the tuning cache's entry, else the
 *     built-in shape), always in its direct-load form: the bulk-copy ring
 *     depth of a fixed tuning is ignored, so the launch has no bounded wait
 *     and no device error word to report.  This call never runs the
 *     first-use tuning search (kf_set_autotune); results may differ from
 *     kf_bicgk's in rounding when the two take different kernel shapes.
 *   - All calls on a device share the array: calls that overlap on the GPU
 *     (unordered streams, concurrent threads) race.  Order them on one
 *     stream.
 * ---------------------------------------------------------------------- */
#define KF_BICGK_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)
kf_status kf_bicgk_noalloc(int64_t m, int64_t n, const float* A, int64_t lda, const float* p,
                           const float* r, float* q, float* s, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* KF_H */
