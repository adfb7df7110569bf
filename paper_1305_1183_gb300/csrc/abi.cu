// C ABI of libkf (include/kf.h): argument checks, program assembly for the
// fused sequences and elementaries, workspace layout, error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/kf.h"
#include "kf_internal.h"

namespace kf {

bool atax_single_pass_ok(int64_t m, int64_t n, int64_t lda, const void* A, const void* x, const void* y);
size_t atax_workspace_bytes(int64_t n);
int launch_atax_tuned(const float* A, int64_t lda, int64_t m, int64_t n, const float* x, float* y, float scale,
                      void* ws, size_t ws_bytes, void* stream, const char** why);
bool gemver_single_ok(int64_t n, const float* A, int64_t lda, const float* B, int64_t ldb, const float* const* vecs,
                      int nvec);
int launch_gemver_single(int64_t n, const float* A, int64_t lda, const float* u1, const float* v1, const float* u2,
                         const float* v2, const float* y, const float* z, float alpha, float beta, float* B,
                         int64_t ldb, float* x, float* w, void* ws, size_t ws_bytes, void* stream, const char** why);
bool sgemvt_single_ok(int64_t m, int64_t n, const float* A, int64_t lda, const float* const* vecs, int nvec);
int launch_sgemvt_single(int64_t m, int64_t n, const float* A, int64_t lda, const float* y, const float* z,
                         float alpha, float beta, float* x, float* w, void* ws, size_t ws_bytes, void* stream,
                         const char** why);
bool tune_cache_get_mat(const std::string& k, MatTune* t);
void tune_cache_put_mat(const std::string& k, const MatTune& t);
bool tune_on_first_use(void* stream);
int launch_madd_strided(int64_t m, int64_t n, const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                        int64_t ldc, void* stream, const char** why);
int launch_quantize_rows(const float* A, int64_t lda, int64_t m, int64_t n, int fmt, void* Q,
                         float* scale, void* stream, const char** why);
extern std::atomic<int> g_autotune_reps;

namespace {
thread_local std::string g_err;
MatTune g_tune = {0, 0, 0, 0, 0};  // automatic
std::mutex g_tune_mu;

kf_status fail(kf_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

kf_status from_launch(int rc, const char* why) {
  if (rc == 0) return KF_OK;
  return fail(rc, why ? why : "launch failed");
}

MatTune cur_tune() {
  std::lock_guard<std::mutex> g(g_tune_mu);
  return g_tune;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
}  // namespace

// Records the calling thread's error message (used by the other C files).
const char* set_error_message(const std::string& msg) {
  g_err = msg;
  return g_err.c_str();
}

MatTune current_matrix_tuning();

int device_sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cache[dev] = v;
  }
  return cache[dev];
}

MatTune current_matrix_tuning() { return cur_tune(); }

}  // namespace kf

using namespace kf;

namespace {

bool bad_fmt(int f) { return f != KF_F32 && f != KF_BF16_ROWSCALE && f != KF_FP8E4M3_ROWSCALE; }

MatProg new_prog(int64_t m, int64_t n) {
  MatProg P;
  std::memset(&P, 0, sizeof(P));
  P.m = m;
  P.n = n;
  return P;
}

EpiOut epi1(float* dst, float coef0) {
  EpiOut o;
  std::memset(&o, 0, sizeof(o));
  o.dst = dst;
  o.nterm = 1;
  o.src[0] = 0;
  o.coef[0] = coef0;
  return o;
}

void epi_add_ext(EpiOut& o, const float* ext, float coef) {
  o.src[o.nterm] = -1;
  o.ext[o.nterm] = ext;
  o.coef[o.nterm] = coef;
  o.nterm++;
}

void epi_add_res(EpiOut& o, int res, float coef) {
  o.src[o.nterm] = res;
  o.coef[o.nterm] = coef;
  o.nterm++;
}

MatOp op_gemv(int mat, int res, const float* x) {
  MatOp o{};
  o.kind = MOP_GEMV; o.mat = mat; o.res = res; o.colvec = x;
  return o;
}
MatOp op_gemvt(int mat, int res, const float* y) {
  MatOp o{};
  o.kind = MOP_GEMVT; o.mat = mat; o.res = res; o.rowvec = y;
  return o;
}
MatOp op_ger(int mat, float alpha, const float* u, const float* v) {
  MatOp o{};
  o.kind = MOP_GER; o.mat = mat; o.alpha = alpha; o.rowvec = u; o.colvec = v;
  return o;
}

kf_status run_mat(MatProg& P, void* ws, size_t ws_bytes, void* stream) {
  int rc = matprog_bind_workspace(P, ws, ws_bytes);
  if (rc != 0) return fail(KF_ERR_WORKSPACE, "workspace missing or smaller than kf_workspace_size()");
  const char* why = nullptr;
  rc = launch_matprog(P, cur_tune(), stream, &why);
  return from_launch(rc, why);
}

kf_status run_vec(VecProg& P, void* ws, size_t ws_bytes, void* stream) {
  if (P.ndot > 0) {
    if (ws == nullptr || ws_bytes < vecprog_workspace_bytes(P.ndot))
      return fail(KF_ERR_WORKSPACE, "workspace missing or smaller than kf_workspace_size()");
    P.counter = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + WS_HEADER);
    P.dotpart = reinterpret_cast<float*>(static_cast<char*>(ws) + WS_HEADER + 256);
  }
  P.fp64_final = P.n >= (int64_t(1) << 26);
  const char* why = nullptr;
  VecTune t{0, 0, 0};  // automatic (tuning cache or defaults)
  return from_launch(launch_vecprog(P, t, stream, &why), why);
}

VecProg new_vec(int64_t n) {
  VecProg P;
  std::memset(&P, 0, sizeof(P));
  P.n = n;
  return P;
}

#define REQ(cond, code, msg)                 \
  do {                                       \
    if (!(cond)) return fail((code), (msg)); \
  } while (0)

kf_status check_mat(int64_t m, int64_t n, const void* A, int64_t lda) {
  REQ(m >= 0 && n >= 0, KF_ERR_INVALID_ARG, "negative size");
  REQ(m == 0 || n == 0 || A != nullptr, KF_ERR_INVALID_ARG, "null matrix");
  REQ(m == 0 || lda >= n, KF_ERR_SHAPE, "leading dimension smaller than the row length");
  REQ(m < (int64_t(1) << 40) && n < (int64_t(1) << 40), KF_ERR_SHAPE, "size too large");
  return KF_OK;
}

kf_status check_vec(int64_t len, const void* p, const char* name) {
  if (len > 0 && p == nullptr) return fail(KF_ERR_INVALID_ARG, std::string("null vector ") + name);
  return KF_OK;
}

#define CHK(expr)                     \
  do {                                \
    kf_status _s = (expr);            \
    if (_s != KF_OK) return _s;       \
  } while (0)

}  // namespace

namespace kf {

size_t atax_plan_workspace_bytes(int64_t m, int64_t n) {
  return std::max(atax_workspace_bytes(n),
                  256 + align256((size_t)m * sizeof(float)) + matprog_workspace_bytes(m, n, 1, 1, FMT_F32));
}

// y = scale * A^T (A x).  One read of A when the rows fit the shared-memory
// ring and are 16-byte aligned; else the paper's two passes, t = A x into
// the workspace (after its first 256 bytes, the device error word), then
// y = scale * A^T t.
int atax_run(int64_t m, int64_t n, const float* A, int64_t lda, const float* x, float* y, float scale, void* ws,
             size_t ws_bytes, void* stream) {
  if (n == 0) return KF_OK;
  if (atax_single_pass_ok(m, n, lda, A, x, y)) {
    const char* why = nullptr;
    if (ws == nullptr) return fail(KF_ERR_WORKSPACE, "workspace required");
    return from_launch(launch_atax_tuned(A, lda, m, n, x, y, scale, ws, ws_bytes, stream, &why), why);
  }
  REQ(ws != nullptr, KF_ERR_WORKSPACE, "workspace required");
  float* t = reinterpret_cast<float*>(static_cast<char*>(ws) + 256);
  const size_t toff = 256 + align256((size_t)m * sizeof(float));
  REQ(ws_bytes >= toff, KF_ERR_WORKSPACE, "workspace too small");
  void* ws2 = static_cast<char*>(ws) + toff;
  const size_t ws2b = ws_bytes - toff;
  MatProg P = new_prog(m, n);
  P.nmat = 1; P.fmt = FMT_F32; P.A[0] = A; P.lda[0] = lda;
  P.nops = 1; P.ops[0] = op_gemv(0, 0, x);
  P.nrow_res = 1; P.ncol_res = 1;
  P.nrow_out = m > 0 ? 1 : 0; P.row_out[0] = epi1(t, 1.f);
  if (m > 0) CHK(run_mat(P, ws2, ws2b, stream));
  MatProg Q = new_prog(m, n);
  Q.nmat = 1; Q.fmt = FMT_F32; Q.A[0] = A; Q.lda[0] = lda;
  Q.nops = 1; Q.ops[0] = op_gemvt(0, 0, t);
  Q.nrow_res = 1; Q.ncol_res = 1;
  Q.ncol_out = 1; Q.col_out[0] = epi1(y, scale);
  return run_mat(Q, ws2, ws2b, stream);
}

}  // namespace kf

extern "C" {

const char* kf_version(void) { return "kf 0.1.0 (sm_103a)"; }

const char* kf_last_error(void) { return g_err.c_str(); }

kf_status kf_device_sm_count(int* sm_count) {
  REQ(sm_count != nullptr, KF_ERR_INVALID_ARG, "null output");
  *sm_count = device_sm_count();
  return KF_OK;
}

kf_status kf_workspace_size(kf_seq seq, int64_t m, int64_t n, kf_dtype fmt, size_t* bytes) {
  REQ(bytes != nullptr, KF_ERR_INVALID_ARG, "null output");
  REQ(m >= 0 && n >= 0, KF_ERR_INVALID_ARG, "negative size");
  REQ(!bad_fmt(fmt), KF_ERR_DTYPE, "unknown storage format");
  const int f = (int)fmt;
  switch (seq) {
    case KF_SEQ_BICGK: *bytes = matprog_workspace_bytes(m, n, 1, 1, f); break;
    case KF_SEQ_GEMVER: *bytes = matprog_workspace_bytes(n, n, 1, 1, f); break;
    case KF_SEQ_GESUMMV: *bytes = matprog_workspace_bytes(m, n, 2, 0, f); break;
    case KF_SEQ_ATAX: *bytes = atax_plan_workspace_bytes(m, n); break;
    case KF_SEQ_AXPYDOT:
    case KF_SEQ_DOT: *bytes = vecprog_workspace_bytes(1); break;
    case KF_SEQ_SGEMVT: *bytes = matprog_workspace_bytes(m, n, 1, 1, f); break;
    case KF_SEQ_WAXPBY: *bytes = 0; break;
    case KF_SEQ_GEMV: *bytes = matprog_workspace_bytes(m, n, 1, 0, f); break;
    case KF_SEQ_GEMVT: *bytes = matprog_workspace_bytes(m, n, 0, 1, f); break;
    default: return fail(KF_ERR_INVALID_ARG, "unknown call kind");
  }
  return KF_OK;
}

kf_status kf_workspace_init(void* ws, size_t bytes, void* stream) {
  if (bytes == 0) return KF_OK;
  REQ(ws != nullptr, KF_ERR_INVALID_ARG, "null workspace");
  cudaError_t e = cudaMemsetAsync(ws, 0, bytes, (cudaStream_t)stream);
  REQ(e == cudaSuccess, KF_ERR_CUDA, cudaGetErrorString(e));
  return KF_OK;
}

kf_status kf_workspace_status(void* ws, void* stream) {
  REQ(ws != nullptr, KF_ERR_INVALID_ARG, "null workspace");
  unsigned word = 0;
  cudaError_t e = cudaMemcpyAsync(&word, ws, sizeof(word), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  REQ(e == cudaSuccess, KF_ERR_CUDA, cudaGetErrorString(e));
  if (word & 1u) {
    unsigned zero = 0;
    cudaMemcpy(ws, &zero, sizeof(zero), cudaMemcpyHostToDevice);
    return fail(KF_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out (bulk copy never completed)");
  }
  return KF_OK;
}

kf_status kf_bicgk(int64_t m, int64_t n, const void* A, int64_t lda, kf_dtype fmt,
                   const float* row_scale, const float* p, const float* r, float* q, float* s,
                   void* ws, size_t ws_bytes, void* stream) {
  CHK(check_mat(m, n, A, lda));
  REQ(!bad_fmt(fmt), KF_ERR_DTYPE, "unknown storage format");
  REQ(fmt == KF_F32 || m == 0 || row_scale != nullptr, KF_ERR_INVALID_ARG, "row scales required");
  CHK(check_vec(n, p, "p")); CHK(check_vec(m, r, "r"));
  CHK(check_vec(m, q, "q")); CHK(check_vec(n, s, "s"));
  if (m == 0 && n == 0) return KF_OK;
  MatProg P = new_prog(m, n);
  P.nmat = 1; P.fmt = (int)fmt; P.A[0] = A; P.rscale[0] = row_scale; P.lda[0] = lda;
  P.nops = 2;
  P.ops[0] = op_gemv(0, 0, p);
  P.ops[1] = op_gemvt(0, 0, r);
  P.nrow_res = 1; P.ncol_res = 1;
  P.nrow_out = m > 0 ? 1 : 0; P.row_out[0] = epi1(q, 1.f);
  P.ncol_out = n > 0 ? 1 : 0; P.col_out[0] = epi1(s, 1.f);
  return run_mat(P, ws, ws_bytes, stream);
}

static kf_status gemver_two_pass(int64_t n, const float* A, int64_t lda, const float* u1, const float* v1,
                    const float* u2, const float* v2, const float* y, const float* z, float alpha,
                    float beta, float* B, int64_t ldb, float* x, float* w, void* ws,
                    size_t ws_bytes, void* stream) {
  // Pass 1: B = A + u1 v1^T + u2 v2^T (written once), x = beta B^T y + z.
  MatProg P = new_prog(n, n);
  P.nmat = 1; P.fmt = FMT_F32; P.A[0] = A; P.lda[0] = lda; P.Bout[0] = B; P.ldb[0] = ldb;
  P.nops = 3;
  P.ops[0] = op_ger(0, 1.f, u1, v1);
  P.ops[1] = op_ger(0, 1.f, u2, v2);
  P.ops[2] = op_gemvt(0, 0, y);
  P.nrow_res = 1; P.ncol_res = 1;  // layout shared with pass 2
  P.ncol_out = 1; P.col_out[0] = epi1(x, beta);
  epi_add_ext(P.col_out[0], z, 1.f);
  // B is read again by pass 2: stored at normal L2 priority
  P.l2_keep_out = 1;
  CHK(run_mat(P, ws, ws_bytes, stream));
  // Pass 2 (after the global barrier on x): w = alpha B x, each row group
  // walked from its last rows, the ones pass 1 wrote last (still in L2).
  MatProg Q = new_prog(n, n);
  Q.nmat = 1; Q.fmt = FMT_F32; Q.A[0] = B; Q.lda[0] = ldb;
  Q.reverse_rows = 1;
  Q.nops = 1;
  Q.ops[0] = op_gemv(0, 0, x);
  Q.nrow_res = 1; Q.ncol_res = 1;
  Q.nrow_out = 1; Q.row_out[0] = epi1(w, alpha);
  return run_mat(Q, ws, ws_bytes, stream);
}

static int log2_floor(int64_t v) {
  int b = 0;
  while (b < 62 && (int64_t(1) << (b + 1)) <= v) ++b;
  return b;
}

// The form of a sequence with a one-launch and a two-launch implementation,
// by the tuning cache (key: warps 1 = one launch, 2 = two); on a miss with
// tuning on first use, both forms are timed on the call's operands (mean of
// `reps` back-to-back calls, best of two rounds, after one run of the
// two-launch form that lets its passes tune) and the one launch kept only if
// it gains more than 2 %; else the two-launch form.
extern "C++" {
template <class Two, class One>
static int choose_form(const std::string& key, void* stream, Two two, One one) {
  MatTune t{};
  if (tune_cache_get_mat(key, &t)) return t.warps == 1 ? 1 : 2;
  if (!tune_on_first_use(stream)) return 2;
  cudaStream_t st = (cudaStream_t)stream;
  const int reps = std::max(1, g_autotune_reps.load());
  if (two() != KF_OK) return 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best[3] = {0.f, 1e30f, 1e30f};
  kf_status rc = KF_OK;
  for (int f : {2, 1, 2, 1}) {
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && rc == KF_OK; ++r) rc = f == 2 ? two() : one();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best[f] = std::min(best[f], ms / (float)reps);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != KF_OK) return 2;
  const int form = best[1] < 0.98f * best[2] ? 1 : 2;
  tune_cache_put_mat(key, MatTune{form, 0, 0, 0, 0});
  return form;
}
}  // extern "C++"

static kf_status check_gemver(int64_t n, const float* A, int64_t lda, const float* u1, const float* v1,
                       const float* u2, const float* v2, const float* y, const float* z, float* B, int64_t ldb,
                       float* x, float* w) {
  CHK(check_mat(n, n, A, lda));
  CHK(check_mat(n, n, B, ldb));
  CHK(check_vec(n, u1, "u1")); CHK(check_vec(n, v1, "v1")); CHK(check_vec(n, u2, "u2"));
  CHK(check_vec(n, v2, "v2")); CHK(check_vec(n, y, "y")); CHK(check_vec(n, z, "z"));
  CHK(check_vec(n, x, "x")); CHK(check_vec(n, w, "w"));
  REQ((const void*)B != (const void*)A || ldb == lda, KF_ERR_SHAPE, "in-place B needs ldb == lda");
  return KF_OK;
}

kf_status kf_gemver_single(int64_t n, const float* A, int64_t lda, const float* u1, const float* v1,
                           const float* u2, const float* v2, const float* y, const float* z, float alpha,
                           float beta, float* B, int64_t ldb, float* x, float* w, void* ws, size_t ws_bytes,
                           void* stream) {
  CHK(check_gemver(n, A, lda, u1, v1, u2, v2, y, z, B, ldb, x, w));
  if (n == 0) return KF_OK;
  const float* vecs[8] = {u1, v1, u2, v2, y, z, x, w};
  REQ(gemver_single_ok(n, A, lda, B, ldb, vecs, 8), KF_ERR_UNSUPPORTED,
      "the single launch needs n a multiple of 4 (n >= 8), 16-byte aligned operands and B not in place of A");
  const char* why = nullptr;
  return from_launch(launch_gemver_single(n, A, lda, u1, v1, u2, v2, y, z, alpha, beta, B, ldb, x, w, ws, ws_bytes,
                                          stream, &why), why);
}

kf_status kf_gemver(int64_t n, const float* A, int64_t lda, const float* u1, const float* v1,
                    const float* u2, const float* v2, const float* y, const float* z, float alpha,
                    float beta, float* B, int64_t ldb, float* x, float* w, void* ws,
                    size_t ws_bytes, void* stream) {
  CHK(check_gemver(n, A, lda, u1, v1, u2, v2, y, z, B, ldb, x, w));
  if (n == 0) return KF_OK;
  const float* vecs[8] = {u1, v1, u2, v2, y, z, x, w};
  const bool single_ok = gemver_single_ok(n, A, lda, B, ldb, vecs, 8) && ws != nullptr &&
                         ws_bytes >= matprog_workspace_bytes(n, n, 1, 1, FMT_F32) && cur_tune().warps == 0;
  auto two = [&]() {
    return gemver_two_pass(n, A, lda, u1, v1, u2, v2, y, z, alpha, beta, B, ldb, x, w, ws, ws_bytes, stream);
  };
  auto one = [&]() {
    return kf_gemver_single(n, A, lda, u1, v1, u2, v2, y, z, alpha, beta, B, ldb, x, w, ws, ws_bytes, stream);
  };
  const int form = single_ok ? choose_form("gemver_form " + std::to_string(log2_floor(n)), stream, two, one) : 2;
  if (form == 1)
    return kf_gemver_single(n, A, lda, u1, v1, u2, v2, y, z, alpha, beta, B, ldb, x, w, ws, ws_bytes, stream);
  return gemver_two_pass(n, A, lda, u1, v1, u2, v2, y, z, alpha, beta, B, ldb, x, w, ws, ws_bytes, stream);
}

kf_status kf_gemver_q(int64_t n, const void* QA, int64_t lda, kf_dtype fmt, const float* sA, const float* u1,
                      const float* v1, const float* u2, const float* v2, const float* y, const float* z,
                      float alpha, float beta, void* QB, int64_t ldb, float* sB, float* x, float* w, void* ws,
                      size_t ws_bytes, void* stream) {
  REQ(fmt == KF_BF16_ROWSCALE || fmt == KF_FP8E4M3_ROWSCALE, KF_ERR_DTYPE, "kf_gemver_q takes BF16 or E4M3 codes");
  CHK(check_mat(n, n, QA, lda));
  CHK(check_mat(n, n, QB, ldb));
  REQ(n == 0 || (sA != nullptr && sB != nullptr), KF_ERR_INVALID_ARG, "row scales required");
  CHK(check_vec(n, u1, "u1")); CHK(check_vec(n, v1, "v1")); CHK(check_vec(n, u2, "u2"));
  CHK(check_vec(n, v2, "v2")); CHK(check_vec(n, y, "y")); CHK(check_vec(n, z, "z"));
  CHK(check_vec(n, x, "x")); CHK(check_vec(n, w, "w"));
  REQ(QB != QA, KF_ERR_SHAPE, "QB must not alias QA");
  if (n == 0) return KF_OK;
  REQ(ws != nullptr && ws_bytes >= WS_HEADER, KF_ERR_WORKSPACE, "workspace required");
  // max |v1|, max |v2| for the row-scale bound, in the workspace header
  float* norms = reinterpret_cast<float*>(static_cast<char*>(ws) + WS_AUX);
  // Pass 1: B = Ahat + u1 v1^T + u2 v2^T stored as codes + row scales,
  // x = beta Bhat^T y + z.
  MatProg P = new_prog(n, n);
  P.nmat = 1; P.fmt = (int)fmt; P.A[0] = QA; P.rscale[0] = sA; P.lda[0] = lda;
  P.Bout[0] = static_cast<float*>(QB); P.ldb[0] = ldb; P.Bscale[0] = sB;
  P.nops = 3;
  P.ops[0] = op_ger(0, 1.f, u1, v1); P.ops[0].vnorm = norms;
  P.ops[1] = op_ger(0, 1.f, u2, v2); P.ops[1].vnorm = norms + 1;
  P.ops[2] = op_gemvt(0, 0, y);
  P.nrow_res = 1; P.ncol_res = 1;
  P.ncol_out = 1; P.col_out[0] = epi1(x, beta);
  epi_add_ext(P.col_out[0], z, 1.f);
  {
    // the passes' workspace rule, checked before the norm pre-pass is enqueued
    MatProg chk = P;
    if (matprog_bind_workspace(chk, ws, ws_bytes) != 0)
      return fail(KF_ERR_WORKSPACE, "workspace missing or smaller than kf_workspace_size()");
  }
  const float* vs[2] = {v1, v2};
  const char* why = nullptr;
  CHK(from_launch(launch_colnorms(vs, 2, n, norms, stream, &why), why));
  P.l2_keep_out = 1;  // as kf_gemver: QB stays in L2 for pass 2
  CHK(run_mat(P, ws, ws_bytes, stream));
  // Pass 2: w = alpha Bhat x, rows walked from those written last.
  MatProg Q = new_prog(n, n);
  Q.nmat = 1; Q.fmt = (int)fmt; Q.A[0] = QB; Q.rscale[0] = sB; Q.lda[0] = ldb;
  Q.reverse_rows = 1;
  Q.nops = 1;
  Q.ops[0] = op_gemv(0, 0, x);
  Q.nrow_res = 1; Q.ncol_res = 1;
  Q.nrow_out = 1; Q.row_out[0] = epi1(w, alpha);
  return run_mat(Q, ws, ws_bytes, stream);
}

static kf_status sgemvt_two_pass(int64_t m, int64_t n, const float* A, int64_t lda, const float* y, const float* z,
                     float alpha, float beta, float* x, float* w, void* ws, size_t ws_bytes, void* stream) {
  // Pass 1: x = beta A^T y + z.
  MatProg P = new_prog(m, n);
  P.nmat = 1; P.fmt = FMT_F32; P.A[0] = A; P.lda[0] = lda;
  P.nops = 1;
  P.ops[0] = op_gemvt(0, 0, y);
  P.nrow_res = 1; P.ncol_res = 1;  // layout shared with pass 2
  P.ncol_out = n > 0 ? 1 : 0; P.col_out[0] = epi1(x, beta);
  epi_add_ext(P.col_out[0], z, 1.f);
  CHK(run_mat(P, ws, ws_bytes, stream));
  if (m == 0) return KF_OK;
  // Pass 2 (after the global barrier on x): w = alpha A x, each row group
  // walked from its last rows (the likeliest still in L2).
  MatProg Q = new_prog(m, n);
  Q.nmat = 1; Q.fmt = FMT_F32; Q.A[0] = A; Q.lda[0] = lda;
  Q.reverse_rows = 1;
  Q.nops = 1;
  Q.ops[0] = op_gemv(0, 0, x);
  Q.nrow_res = 1; Q.ncol_res = 1;
  Q.nrow_out = 1; Q.row_out[0] = epi1(w, alpha);
  return run_mat(Q, ws, ws_bytes, stream);
}

kf_status kf_sgemvt_single(int64_t m, int64_t n, const float* A, int64_t lda, const float* y, const float* z,
                           float alpha, float beta, float* x, float* w, void* ws, size_t ws_bytes, void* stream) {
  CHK(check_mat(m, n, A, lda));
  CHK(check_vec(m, y, "y")); CHK(check_vec(n, z, "z"));
  CHK(check_vec(n, x, "x")); CHK(check_vec(m, w, "w"));
  if (m == 0 && n == 0) return KF_OK;
  const float* vecs[4] = {y, z, x, w};
  REQ(sgemvt_single_ok(m, n, A, lda, vecs, 4), KF_ERR_UNSUPPORTED,
      "the single launch needs m >= 8, n a multiple of 4 and 16-byte aligned operands");
  const char* why = nullptr;
  return from_launch(launch_sgemvt_single(m, n, A, lda, y, z, alpha, beta, x, w, ws, ws_bytes, stream, &why), why);
}

kf_status kf_sgemvt(int64_t m, int64_t n, const float* A, int64_t lda, const float* y, const float* z,
                    float alpha, float beta, float* x, float* w, void* ws, size_t ws_bytes, void* stream) {
  CHK(check_mat(m, n, A, lda));
  CHK(check_vec(m, y, "y")); CHK(check_vec(n, z, "z"));
  CHK(check_vec(n, x, "x")); CHK(check_vec(m, w, "w"));
  if (m == 0 && n == 0) return KF_OK;
  const float* vecs[4] = {y, z, x, w};
  const bool single_ok = sgemvt_single_ok(m, n, A, lda, vecs, 4) && ws != nullptr &&
                         ws_bytes >= matprog_workspace_bytes(m, n, 1, 1, FMT_F32) && cur_tune().warps == 0;
  auto two = [&]() { return sgemvt_two_pass(m, n, A, lda, y, z, alpha, beta, x, w, ws, ws_bytes, stream); };
  auto one = [&]() { return kf_sgemvt_single(m, n, A, lda, y, z, alpha, beta, x, w, ws, ws_bytes, stream); };
  const int form = single_ok ? choose_form("sgemvt_form " + std::to_string(log2_floor(m)) + " " +
                                               std::to_string(log2_floor(n)), stream, two, one)
                             : 2;
  return form == 1 ? one() : two();
}

kf_status kf_gesummv(int64_t m, int64_t n, const float* A, const float* B, int64_t lda,
                     const float* x, float alpha, float beta, float* y, void* ws, size_t ws_bytes,
                     void* stream) {
  CHK(check_mat(m, n, A, lda));
  CHK(check_mat(m, n, B, lda));
  CHK(check_vec(n, x, "x")); CHK(check_vec(m, y, "y"));
  if (m == 0) return KF_OK;
  MatProg P = new_prog(m, n);
  P.nmat = 2; P.fmt = FMT_F32;
  P.A[0] = A; P.lda[0] = lda; P.A[1] = B; P.lda[1] = lda;
  P.nops = 2;
  P.ops[0] = op_gemv(0, 0, x);
  P.ops[1] = op_gemv(1, 1, x);
  P.nrow_res = 2; P.ncol_res = 0;
  P.nrow_out = 1; P.row_out[0] = epi1(y, alpha);
  epi_add_res(P.row_out[0], 1, beta);
  return run_mat(P, ws, ws_bytes, stream);
}

kf_status kf_atax(int64_t m, int64_t n, const float* A, int64_t lda, const float* x, float* y,
                  void* ws, size_t ws_bytes, void* stream) {
  CHK(check_mat(m, n, A, lda));
  CHK(check_vec(n, x, "x")); CHK(check_vec(n, y, "y"));
  if (n == 0) return KF_OK;
  return kf::atax_run(m, n, A, lda, x, y, 1.f, ws, ws_bytes, stream);
}

kf_status kf_axpydot(int64_t n, const float* w, const float* v, const float* u, float alpha,
                     float* z, float* r, void* ws, size_t ws_bytes, void* stream) {
  REQ(n >= 0, KF_ERR_INVALID_ARG, "negative size");
  CHK(check_vec(n, w, "w")); CHK(check_vec(n, v, "v")); CHK(check_vec(n, u, "u"));
  CHK(check_vec(n, z, "z"));
  REQ(r != nullptr, KF_ERR_INVALID_ARG, "null r");
  VecProg P = new_vec(n);
  P.nin = 3; P.in[0] = w; P.in[1] = v; P.in[2] = u;
  P.nout = 1; P.out[0] = z; P.C[0][0] = 1.f; P.C[0][1] = -alpha; P.C[0][2] = 0.f;
  P.ndot = 1; P.dot_out[0] = r;
  P.P[0][0] = 1.f; P.P[0][1] = -alpha; P.P[0][2] = 0.f;
  P.Q[0][0] = 0.f; P.Q[0][1] = 0.f; P.Q[0][2] = 1.f;
  return run_vec(P, ws, ws_bytes, stream);
}

kf_status kf_waxpby(int64_t n, float alpha, const float* x, float beta, const float* y, float* w,
                    void* stream) {
  REQ(n >= 0, KF_ERR_INVALID_ARG, "negative size");
  CHK(check_vec(n, x, "x")); CHK(check_vec(n, y, "y")); CHK(check_vec(n, w, "w"));
  if (n == 0) return KF_OK;
  VecProg P = new_vec(n);
  P.nin = 2; P.in[0] = x; P.in[1] = y;
  P.nout = 1; P.out[0] = w; P.C[0][0] = alpha; P.C[0][1] = beta;
  return run_vec(P, nullptr, 0, stream);
}

kf_status kf_gemv(int64_t m, int64_t n, const void* A, int64_t lda, kf_dtype fmt,
                  const float* row_scale, float alpha, const float* x, float beta,
                  const float* y0, float* y, void* ws, size_t ws_bytes, void* stream) {
  CHK(check_mat(m, n, A, lda));
  REQ(!bad_fmt(fmt), KF_ERR_DTYPE, "unknown storage format");
  REQ(fmt == KF_F32 || m == 0 || row_scale != nullptr, KF_ERR_INVALID_ARG, "row scales required");
  CHK(check_vec(n, x, "x")); CHK(check_vec(m, y, "y"));
  REQ(beta == 0.f || m == 0 || y0 != nullptr, KF_ERR_INVALID_ARG, "null y0 with beta != 0");
  if (m == 0) return KF_OK;
  MatProg P = new_prog(m, n);
  P.nmat = 1; P.fmt = (int)fmt; P.A[0] = A; P.rscale[0] = row_scale; P.lda[0] = lda;
  P.nops = 1; P.ops[0] = op_gemv(0, 0, x);
  P.nrow_res = 1; P.ncol_res = 0;
  P.nrow_out = 1; P.row_out[0] = epi1(y, alpha);
  if (beta != 0.f) epi_add_ext(P.row_out[0], y0, beta);
  return run_mat(P, ws, ws_bytes, stream);
}

kf_status kf_gemvt(int64_t m, int64_t n, const void* A, int64_t lda, kf_dtype fmt,
                   const float* row_scale, float alpha, const float* y, float beta,
                   const float* x0, float* x, void* ws, size_t ws_bytes, void* stream) {
  CHK(check_mat(m, n, A, lda));
  REQ(!bad_fmt(fmt), KF_ERR_DTYPE, "unknown storage format");
  REQ(fmt == KF_F32 || m == 0 || row_scale != nullptr, KF_ERR_INVALID_ARG, "row scales required");
  CHK(check_vec(m, y, "y")); CHK(check_vec(n, x, "x"));
  REQ(beta == 0.f || n == 0 || x0 != nullptr, KF_ERR_INVALID_ARG, "null x0 with beta != 0");
  if (n == 0) return KF_OK;
  MatProg P = new_prog(m, n);
  P.nmat = 1; P.fmt = (int)fmt; P.A[0] = A; P.rscale[0] = row_scale; P.lda[0] = lda;
  P.nops = 1; P.ops[0] = op_gemvt(0, 0, y);
  P.nrow_res = 0; P.ncol_res = 1;
  P.ncol_out = 1; P.col_out[0] = epi1(x, alpha);
  if (beta != 0.f) epi_add_ext(P.col_out[0], x0, beta);
  return run_mat(P, ws, ws_bytes, stream);
}

kf_status kf_ger(int64_t m, int64_t n, const float* A, int64_t lda, float alpha, const float* u,
                 const float* v, float* B, int64_t ldb, void* stream) {
  CHK(check_mat(m, n, A, lda));
  CHK(check_mat(m, n, B, ldb));
  CHK(check_vec(m, u, "u")); CHK(check_vec(n, v, "v"));
  REQ((const void*)B != (const void*)A || ldb == lda, KF_ERR_SHAPE, "in-place B needs ldb == lda");
  if (m == 0 || n == 0) return KF_OK;
  MatProg P = new_prog(m, n);
  P.nmat = 1; P.fmt = FMT_F32; P.A[0] = A; P.lda[0] = lda; P.Bout[0] = B; P.ldb[0] = ldb;
  P.nops = 1; P.ops[0] = op_ger(0, alpha, u, v);
  return run_mat(P, nullptr, 0, stream);
}

kf_status kf_axpby(int64_t n, float alpha, const float* x, float beta, const float* y, float* out,
                   void* stream) {
  REQ(n >= 0, KF_ERR_INVALID_ARG, "negative size");
  CHK(check_vec(n, x, "x")); CHK(check_vec(n, out, "out"));
  REQ(beta == 0.f || n == 0 || y != nullptr, KF_ERR_INVALID_ARG, "null y with beta != 0");
  if (n == 0) return KF_OK;
  VecProg P = new_vec(n);
  P.nin = beta != 0.f ? 2 : 1; P.in[0] = x; P.in[1] = y;
  P.nout = 1; P.out[0] = out; P.C[0][0] = alpha; P.C[0][1] = beta;
  return run_vec(P, nullptr, 0, stream);
}

kf_status kf_scal(int64_t n, float alpha, const float* x, float* out, void* stream) {
  REQ(n >= 0, KF_ERR_INVALID_ARG, "negative size");
  CHK(check_vec(n, x, "x")); CHK(check_vec(n, out, "out"));
  if (n == 0) return KF_OK;
  VecProg P = new_vec(n);
  P.nin = 1; P.in[0] = x;
  P.nout = 1; P.out[0] = out; P.C[0][0] = alpha;
  return run_vec(P, nullptr, 0, stream);
}

kf_status kf_vadd3(int64_t n, const float* w, const float* y, const float* z, float* out,
                   void* stream) {
  REQ(n >= 0, KF_ERR_INVALID_ARG, "negative size");
  CHK(check_vec(n, w, "w")); CHK(check_vec(n, y, "y")); CHK(check_vec(n, z, "z"));
  CHK(check_vec(n, out, "out"));
  if (n == 0) return KF_OK;
  VecProg P = new_vec(n);
  P.nin = 3; P.in[0] = w; P.in[1] = y; P.in[2] = z;
  P.nout = 1; P.out[0] = out; P.C[0][0] = 1.f; P.C[0][1] = 1.f; P.C[0][2] = 1.f;
  return run_vec(P, nullptr, 0, stream);
}

kf_status kf_madd(int64_t m, int64_t n, const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                  int64_t ldc, void* stream) {
  CHK(check_mat(m, n, A, lda));
  CHK(check_mat(m, n, B, ldb));
  CHK(check_mat(m, n, C, ldc));
  if (m == 0 || n == 0) return KF_OK;
  if (lda == n && ldb == n && ldc == n) {
    // contiguous: one vector pass over m n elements
    VecProg P = new_vec(m * n);
    P.nin = 2; P.in[0] = A; P.in[1] = B;
    P.nout = 1; P.out[0] = C; P.C[0][0] = 1.f; P.C[0][1] = 1.f;
    return run_vec(P, nullptr, 0, stream);
  }
  const char* why = nullptr;
  return from_launch(launch_madd_strided(m, n, A, lda, B, ldb, C, ldc, stream, &why), why);
}

kf_status kf_dot(int64_t n, const float* x, const float* y, float* out, void* ws, size_t ws_bytes,
                 void* stream) {
  REQ(n >= 0, KF_ERR_INVALID_ARG, "negative size");
  CHK(check_vec(n, x, "x")); CHK(check_vec(n, y, "y"));
  REQ(out != nullptr, KF_ERR_INVALID_ARG, "null out");
  VecProg P = new_vec(n);
  P.nin = 2; P.in[0] = x; P.in[1] = y;
  P.nout = 0;
  P.ndot = 1; P.dot_out[0] = out;
  P.P[0][0] = 1.f; P.P[0][1] = 0.f; P.Q[0][0] = 0.f; P.Q[0][1] = 1.f;
  return run_vec(P, ws, ws_bytes, stream);
}

kf_status kf_quantize_rows(int64_t m, int64_t n, const float* A, int64_t lda, kf_dtype fmt, void* Q,
                           float* row_scale, void* stream) {
  CHK(check_mat(m, n, A, lda));
  REQ(fmt == KF_BF16_ROWSCALE || fmt == KF_FP8E4M3_ROWSCALE, KF_ERR_DTYPE, "quantised format expected");
  REQ(m == 0 || (Q != nullptr && row_scale != nullptr), KF_ERR_INVALID_ARG, "null output");
  const char* why = nullptr;
  return from_launch(launch_quantize_rows(A, lda, m, n, (int)fmt, Q, row_scale, stream, &why), why);
}

kf_status kf_set_autotune(int reps) {
  REQ(reps >= 0 && reps <= 100, KF_ERR_INVALID_ARG, "reps must be in 0..100");
  g_autotune_reps.store(reps);
  return KF_OK;
}

kf_status kf_get_autotune(int* reps) {
  REQ(reps != nullptr, KF_ERR_INVALID_ARG, "null output");
  *reps = g_autotune_reps.load();
  return KF_OK;
}

kf_status kf_set_matrix_tuning(int warps, int vec, int unroll, int groups, int stages) {
  if (warps == 0) {  // back to the automatic choice
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune = MatTune{0, 0, 0, 0, 0};
    return KF_OK;
  }
  REQ(warps == 4 || warps == 8, KF_ERR_INVALID_ARG, "warps must be 4 or 8 (0 = automatic)");
  REQ(vec == 1 || vec == 2 || vec == 4, KF_ERR_INVALID_ARG, "vec must be 1, 2 or 4");
  REQ(unroll == 1 || unroll == 2 || unroll == 4 || unroll == 8, KF_ERR_INVALID_ARG, "unroll must be 1, 2, 4 or 8");
  REQ(groups >= 0 && groups <= MAT_MAXGROUPS, KF_ERR_INVALID_ARG, "groups out of range");
  REQ(stages >= 0 && stages <= MAT_MAXSTAGES, KF_ERR_INVALID_ARG, "stages out of range");
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune = MatTune{warps, vec, unroll, groups, stages};
  return KF_OK;
}

kf_status kf_get_matrix_tuning(int* warps, int* vec, int* unroll, int* groups, int* stages) {
  REQ(warps && vec && unroll && groups && stages, KF_ERR_INVALID_ARG, "null output");
  MatTune t = cur_tune();
  *warps = t.warps; *vec = t.vec; *unroll = t.unroll; *groups = t.groups; *stages = t.stages;
  return KF_OK;
}

}  // extern "C"
