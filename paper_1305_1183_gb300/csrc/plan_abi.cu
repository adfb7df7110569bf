// C ABI of scripts and plans (include/kf.h, "Scripts and plans").
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/kf.h"
#include "kf_internal.h"
#include "planner.h"

namespace kf {
const char* set_error_message(const std::string& msg);
MatTune current_matrix_tuning();
int autotune_matprog(MatProg& P, void* stream, int reps, MatTune* best, float* best_ms, float* auto_ms);
int autotune_vecprog(VecProg& P, void* stream, int reps, VecTune* best, float* best_ms, float* auto_ms);
void tune_cache_clear();
void tune_cache_dump(std::vector<std::string>* lines);
size_t tune_cache_size();
void tune_cache_put_mat(const std::string& k, const MatTune& t);
void tune_cache_put_vec(const std::string& k, const VecTune& t);
namespace plan {
void set_model(double bw_bytes_per_s, double launch_us);
void get_model(double* bw, double* launch_us);
}  // namespace plan
}  // namespace kf

struct kf_script {
  kf::plan::Script s;
};
struct kf_plan {
  kf::plan::Plan p;
  int nvars = 0;
};

using namespace kf;
using namespace kf::plan;

namespace {

kf_status err(kf_status st, const std::string& m) {
  set_error_message(m);
  return st;
}

kf_status add_var(kf_script* sc, const char* name, int kind, int64_t m, int64_t n, int* id) {
  if (sc == nullptr || id == nullptr) return err(KF_ERR_INVALID_ARG, "null argument");
  if (m < 0 || n < 0) return err(KF_ERR_INVALID_ARG, "negative size");
  Var v;
  v.name = name ? name : ("v" + std::to_string(sc->s.vars.size()));
  v.kind = kind;
  v.m = m;
  v.n = n;
  v.ld = n;
  sc->s.vars.push_back(v);
  sc->s.analysed = false;
  *id = (int)sc->s.vars.size() - 1;
  return KF_OK;
}

kf_status ensure_analysed(const kf_script* sc) {
  auto* s = const_cast<Script*>(&sc->s);
  if (s->analysed) return KF_OK;
  std::string e = analyse(*s);
  if (!e.empty()) {
    const bool undef = e.find("read before") != std::string::npos;
    return err(undef ? KF_ERR_UNDEFINED_VAR : KF_ERR_SHAPE, e);
  }
  return KF_OK;
}

std::vector<std::vector<int>> unfused_groups(const Script& s) {
  std::vector<std::vector<int>> g;
  for (int c = 0; c < (int)s.calls.size(); ++c) g.push_back({c});
  return g;
}

// A plan's workspace: [vector-pass region (header, counter, dot partials) |
// matrix-pass region (its own header, counters, partials)], so that the
// partial sums of one kind never land on the counters of the other.
size_t plan_vec_region() { return (vecprog_workspace_bytes(VP_MAXDOT) + 255) & ~(size_t)255; }

// Bind variable pointers into a copy of a kernel's program and launch it.
kf_status launch_kernel(const Kernel& K, void* const* bindings, int nb, void* ws, size_t ws_bytes, void* stream,
                        const MatTune& tune) {
  if (K.is_atax) {
    void* p[3] = {nullptr, nullptr, nullptr};
    for (auto& b : K.bind) {
      if (b.second < 0 || b.second >= nb || bindings[b.second] == nullptr)
        return err(KF_ERR_INVALID_ARG, "variable " + std::to_string(b.second) + " is not bound");
      p[(size_t)(uintptr_t)b.first] = bindings[b.second];
    }
    char* wsm = ws ? static_cast<char*>(ws) + plan_vec_region() : nullptr;
    const size_t wsm_bytes = ws_bytes > plan_vec_region() ? ws_bytes - plan_vec_region() : 0;
    return atax_run(K.m, K.n, static_cast<const float*>(p[0]), K.lda, static_cast<const float*>(p[1]),
                    static_cast<float*>(p[2]), K.atax_scale, wsm, wsm_bytes, stream);
  }
  if (K.is_mat) {
    MatProg P = K.mp;
    for (auto& b : K.bind) {
      if (b.second < 0 || b.second >= nb || bindings[b.second] == nullptr)
        return err(KF_ERR_INVALID_ARG, "variable " + std::to_string(b.second) + " is not bound");
      *reinterpret_cast<void**>(reinterpret_cast<char*>(&P) + (size_t)(uintptr_t)b.first) = bindings[b.second];
    }
    // matrix passes use the workspace after the vector passes' region
    char* wsm = ws ? static_cast<char*>(ws) + plan_vec_region() : nullptr;
    const size_t wsm_bytes = ws_bytes > plan_vec_region() ? ws_bytes - plan_vec_region() : 0;
    if (P.nrow_res == 0 && P.ncol_res == 0 && P.nrow_out == 0 && P.ncol_out == 0) {
      P.errword = nullptr;
    } else if (matprog_bind_workspace(P, wsm, wsm_bytes) != 0) {
      return err(KF_ERR_WORKSPACE, "workspace missing or smaller than kf_plan_workspace_size()");
    }
    const char* why = nullptr;
    const int rc = launch_matprog(P, tune, stream, &why);
    return rc == 0 ? KF_OK : err(rc, why ? why : "launch failed");
  }
  VecProg P = K.vp;
  for (auto& b : K.bind) {
    if (b.second < 0 || b.second >= nb || bindings[b.second] == nullptr)
      return err(KF_ERR_INVALID_ARG, "variable " + std::to_string(b.second) + " is not bound");
    *reinterpret_cast<void**>(reinterpret_cast<char*>(&P) + (size_t)(uintptr_t)b.first) = bindings[b.second];
  }
  if (P.ndot > 0) {
    if (ws == nullptr || ws_bytes < plan_vec_region())
      return err(KF_ERR_WORKSPACE, "workspace missing or smaller than kf_plan_workspace_size()");
    P.counter = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + WS_HEADER);
    P.dotpart = reinterpret_cast<float*>(static_cast<char*>(ws) + WS_HEADER + 256);
  }
  P.fp64_final = P.n >= (int64_t(1) << 26);
  const char* why = nullptr;
  VecTune t{0, 0, 0};  // automatic (tuning cache or defaults)
  const int rc = launch_vecprog(P, t, stream, &why);
  return rc == 0 ? KF_OK : err(rc, why ? why : "launch failed");
}


// The checks launch_kernel makes, without launching: every variable the
// kernel uses is bound, and the workspace holds what the kernel needs (the
// matrix-pass rule is matprog_bind_workspace's own, on a copy).
kf_status check_kernel(const Kernel& K, void* const* bindings, int nb, void* ws, size_t ws_bytes) {
  for (auto& b : K.bind)
    if (b.second < 0 || b.second >= nb || bindings[b.second] == nullptr)
      return err(KF_ERR_INVALID_ARG, "variable " + std::to_string(b.second) + " is not bound");
  if (K.is_atax) {
    const size_t need = plan_vec_region() + atax_plan_workspace_bytes(K.m, K.n);
    if (ws == nullptr || ws_bytes < need)
      return err(KF_ERR_WORKSPACE, "workspace missing or smaller than kf_plan_workspace_size()");
  } else if (K.is_mat) {
    MatProg P = K.mp;
    char* wsm = ws ? static_cast<char*>(ws) + plan_vec_region() : nullptr;
    const size_t wsm_bytes = ws_bytes > plan_vec_region() ? ws_bytes - plan_vec_region() : 0;
    if (matprog_bind_workspace(P, wsm, wsm_bytes) != 0)
      return err(KF_ERR_WORKSPACE, "workspace missing or smaller than kf_plan_workspace_size()");
  } else if (K.vp.ndot > 0 && (ws == nullptr || ws_bytes < plan_vec_region())) {
    return err(KF_ERR_WORKSPACE, "workspace missing or smaller than kf_plan_workspace_size()");
  }
  return KF_OK;
}

// Every kernel of a plan checked before the first launch, so that a call
// with a missing binding or a short workspace launches nothing.
kf_status check_plan(const Plan& P, void* const* bindings, int nb, void* ws, size_t ws_bytes) {
  for (const Kernel& K : P.kernels) {
    kf_status st = check_kernel(K, bindings, nb, ws, ws_bytes);
    if (st != KF_OK) return st;
  }
  return KF_OK;
}

// Run once, then time `reps` executions with CUDA events; the median (ms).
kf_status time_plan(const Plan& P, int nvars, void* const* bindings, int nb, void* ws, size_t ws_bytes, void* stream,
                    int reps, float* median_ms) {
  if (nb > 0 && bindings == nullptr) return err(KF_ERR_INVALID_ARG, "null bindings");
  if (nb < nvars) return err(KF_ERR_INVALID_ARG, "every script variable needs a binding");
  {
    kf_status chk = check_plan(P, bindings, nb, ws, ws_bytes);
    if (chk != KF_OK) return chk;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const MatTune tune = current_matrix_tuning();
  auto run = [&]() -> kf_status {
    for (const Kernel& K : P.kernels) {
      kf_status rc = launch_kernel(K, bindings, nb, ws, ws_bytes, stream, tune);
      if (rc != KF_OK) return rc;
    }
    return KF_OK;
  };
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return err(KF_ERR_CUDA, "cudaEventCreate failed");
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return err(KF_ERR_CUDA, "cudaEventCreate failed");
  }
  kf_status rc = run();  // warm up
  std::vector<float> t;
  for (int r = 0; r < reps && rc == KF_OK; ++r) {
    cudaEventRecord(a, st);
    rc = run();
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess) rc = err(KF_ERR_CUDA, "timing failed");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    t.push_back(ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != KF_OK) return rc;
  std::sort(t.begin(), t.end());
  *median_ms = t[t.size() / 2];
  return KF_OK;
}

// Name of the program field at byte offset `o` (for plan descriptions).
std::string field_name(const Kernel& K, size_t o) {
  auto at = [&](const void* base, const void* f) { return (size_t)((const char*)f - (const char*)base); };
  if (K.is_atax) return o == 0 ? "A" : o == 1 ? "x" : o == 2 ? "y" : "?";
  if (K.is_mat) {
    const MatProg& P = K.mp;
    for (int t = 0; t < 2; ++t) {
      if (o == at(&P, &P.A[t])) return "A" + std::to_string(t);
      if (o == at(&P, &P.Bout[t])) return "Bout" + std::to_string(t);
    }
    for (int k = 0; k < MAT_MAXOPS; ++k) {
      if (o == at(&P, &P.ops[k].colvec)) return "op" + std::to_string(k) + ".col";
      if (o == at(&P, &P.ops[k].rowvec)) return "op" + std::to_string(k) + ".row";
    }
    for (int j = 0; j < EPI_MAXOUT; ++j) {
      if (o == at(&P, &P.row_out[j].dst)) return "rowout" + std::to_string(j) + ".dst";
      if (o == at(&P, &P.col_out[j].dst)) return "colout" + std::to_string(j) + ".dst";
      for (int t = 0; t < EPI_MAXTERM; ++t) {
        if (o == at(&P, &P.row_out[j].ext[t])) return "rowout" + std::to_string(j) + ".ext";
        if (o == at(&P, &P.col_out[j].ext[t])) return "colout" + std::to_string(j) + ".ext";
      }
    }
    return "?";
  }
  const VecProg& P = K.vp;
  for (int k = 0; k < VP_MAXIN; ++k)
    if (o == at(&P, &P.in[k])) return "in" + std::to_string(k);
  for (int k = 0; k < VP_MAXOUT; ++k)
    if (o == at(&P, &P.out[k])) return "out" + std::to_string(k);
  for (int k = 0; k < VP_MAXDOT; ++k)
    if (o == at(&P, &P.dot_out[k])) return "dot" + std::to_string(k);
  return "?";
}

}  // namespace

extern "C" {

kf_status kf_script_create(kf_script** out) {
  if (out == nullptr) return err(KF_ERR_INVALID_ARG, "null argument");
  *out = new (std::nothrow) kf_script();
  return *out ? KF_OK : err(KF_ERR_NO_MEM, "out of host memory");
}

void kf_script_destroy(kf_script* s) { delete s; }

kf_status kf_script_vector(kf_script* s, const char* name, int64_t n, int* id) {
  return add_var(s, name, VK_VECTOR, 1, n, id);
}

kf_status kf_script_matrix(kf_script* s, const char* name, int64_t m, int64_t n, int* id) {
  return add_var(s, name, VK_MATRIX, m, n, id);
}

kf_status kf_script_matrix_ld(kf_script* s, const char* name, int64_t m, int64_t n, int64_t ld, int* id) {
  if (ld < n || ld < 1) return err(KF_ERR_SHAPE, "matrix row stride ld must be at least n (and at least 1)");
  kf_status st = add_var(s, name, VK_MATRIX, m, n, id);
  if (st == KF_OK) s->s.vars[*id].ld = ld;
  return st;
}

kf_status kf_script_scalar(kf_script* s, const char* name, int* id) { return add_var(s, name, VK_SCALAR, 1, 1, id); }

kf_status kf_script_input(kf_script* s, int id) {
  if (s == nullptr || id < 0 || id >= (int)s->s.vars.size()) return err(KF_ERR_INVALID_ARG, "bad variable id");
  s->s.vars[id].input = true;
  s->s.analysed = false;
  return KF_OK;
}

kf_status kf_script_output(kf_script* s, int id) {
  if (s == nullptr || id < 0 || id >= (int)s->s.vars.size()) return err(KF_ERR_INVALID_ARG, "bad variable id");
  s->s.vars[id].output = true;
  s->s.analysed = false;
  return KF_OK;
}

kf_status kf_script_call(kf_script* s, kf_op op, const int* outs, int n_out, const int* ins, int n_in,
                         const double* scalars, int n_scalars) {
  if (s == nullptr || (n_out > 0 && outs == nullptr) || (n_in > 0 && ins == nullptr) ||
      (n_scalars > 0 && scalars == nullptr) || n_scalars > 2 || n_out < 0 || n_in < 0)
    return err(KF_ERR_INVALID_ARG, "bad call arguments");
  if ((int)op < 0 || (int)op > OP_GER) return err(KF_ERR_INVALID_ARG, "unknown op");
  Call c;
  c.op = (int)op;
  c.outs.assign(outs, outs + n_out);
  c.ins.assign(ins, ins + n_in);
  // defaults: AXPBY (a, b) = (1, 1); SCAL a = 1; GEMV/GEMVT (a, b) = (1, 0 or 1 with y0); GER a = 1
  c.sc[0] = 1.0;
  c.sc[1] = (op == KF_OP_AXPBY) ? 1.0 : ((op == KF_OP_GEMV || op == KF_OP_GEMVT) && n_in == 3 ? 1.0 : 0.0);
  for (int i = 0; i < n_scalars; ++i) c.sc[i] = scalars[i];
  s->s.calls.push_back(c);
  s->s.analysed = false;
  return KF_OK;
}

kf_status kf_script_validate(const kf_script* s) {
  if (s == nullptr) return err(KF_ERR_INVALID_ARG, "null script");
  return ensure_analysed(s);
}

kf_status kf_plan_count(const kf_script* s, int cap, int* count, int* truncated) {
  if (s == nullptr || count == nullptr || cap <= 0) return err(KF_ERR_INVALID_ARG, "bad arguments");
  kf_status st = ensure_analysed(s);
  if (st != KF_OK) return st;
  std::vector<std::vector<std::vector<int>>> all;
  bool tr = false;
  enumerate(s->s, (size_t)cap, &all, &tr);
  *count = (int)all.size();
  if (truncated) *truncated = tr ? 1 : 0;
  return KF_OK;
}

kf_status kf_plan_build(const kf_script* s, const kf_plan_options* opt, kf_plan** out) {
  if (s == nullptr || out == nullptr) return err(KF_ERR_INVALID_ARG, "null argument");
  kf_status st = ensure_analysed(s);
  if (st != KF_OK) return st;
  const int mode = opt ? opt->mode : KF_PLAN_ANALYTIC;
  const int cap = (opt && opt->max_plans > 0) ? opt->max_plans : 20000;
  std::vector<std::vector<int>> chosen;
  if (mode == KF_PLAN_UNFUSED) {
    chosen = unfused_groups(s->s);
  } else {
    std::vector<std::vector<std::vector<int>>> all;
    bool tr = false;
    enumerate(s->s, (size_t)cap, &all, &tr);
    if (all.empty()) return err(KF_ERR_UNSUPPORTED, "no legal plan");
    if (mode == KF_PLAN_INDEX) {
      const int idx = opt ? opt->index : 0;
      if (idx < 0 || idx >= (int)all.size()) return err(KF_ERR_INVALID_ARG, "plan index out of range");
      chosen = all[idx];
    } else if (mode == KF_PLAN_GREEDY) {
      // fewest kernels (fuse as much as legal); first such plan in enumeration order
      size_t best = all[0].size();
      chosen = all[0];
      for (auto& g : all)
        if (g.size() < best) { best = g.size(); chosen = g; }
    } else if (mode == KF_PLAN_ANALYTIC) {
      double best = 1e300;
      for (auto& g : all) {
        Plan p;
        if (!make_plan(s->s, g, &p).empty()) continue;
        if (p.predicted_us < best * (1.0 - 1e-9)) { best = p.predicted_us; chosen = g; }
      }
      if (chosen.empty()) return err(KF_ERR_UNSUPPORTED, "no buildable plan");
    } else {
      return err(KF_ERR_INVALID_ARG, "unknown plan mode");
    }
  }
  auto* pl = new (std::nothrow) kf_plan();
  if (pl == nullptr) return err(KF_ERR_NO_MEM, "out of host memory");
  std::string e = make_plan(s->s, chosen, &pl->p);
  if (!e.empty()) {
    delete pl;
    return err(KF_ERR_UNSUPPORTED, e);
  }
  pl->nvars = (int)s->s.vars.size();
  *out = pl;
  return KF_OK;
}

void kf_plan_destroy(kf_plan* p) { delete p; }

kf_status kf_plan_workspace_size(const kf_plan* p, size_t* bytes) {
  if (p == nullptr || bytes == nullptr) return err(KF_ERR_INVALID_ARG, "null argument");
  *bytes = p->p.ws_bytes;
  return KF_OK;
}

kf_status kf_plan_kernel_count(const kf_plan* p, int* n) {
  if (p == nullptr || n == nullptr) return err(KF_ERR_INVALID_ARG, "null argument");
  *n = (int)p->p.kernels.size();
  return KF_OK;
}

kf_status kf_plan_predicted_us(const kf_plan* p, double* us) {
  if (p == nullptr || us == nullptr) return err(KF_ERR_INVALID_ARG, "null argument");
  *us = p->p.predicted_us;
  return KF_OK;
}

kf_status kf_plan_features(const kf_script* s, const kf_plan* p, float* out, int cap, int* n) {
  if (s == nullptr || p == nullptr || out == nullptr || n == nullptr) return err(KF_ERR_INVALID_ARG, "null argument");
  std::vector<float> f;
  features(s->s, p->p, &f);
  *n = (int)f.size();
  if (cap < (int)f.size()) return err(KF_ERR_INVALID_ARG, "feature buffer too small");
  std::copy(f.begin(), f.end(), out);
  return KF_OK;
}

kf_status kf_plan_describe(const kf_plan* p, char* buf, size_t cap, size_t* needed) {
  if (p == nullptr) return err(KF_ERR_INVALID_ARG, "null plan");
  std::ostringstream o;
  o.precision(17);  // byte counts and predictions round-trip exactly
  o << "{\"predicted_us\":" << p->p.predicted_us << ",\"bytes\":" << p->p.bytes << ",\"kernels\":[";
  for (size_t i = 0; i < p->p.kernels.size(); ++i) {
    const Kernel& K = p->p.kernels[i];
    o << (i ? "," : "") << "{\"kind\":\"" << (K.is_atax ? "atax" : K.is_mat ? "matrix" : "vector") << "\",\"calls\":[";
    for (size_t j = 0; j < K.calls.size(); ++j) o << (j ? "," : "") << K.calls[j];
    o << "]";
    if (K.is_mat) {
      o << ",\"order\":[";
      for (size_t j = 0; j < K.order.size(); ++j) o << (j ? "," : "") << K.order[j];
      o << "],\"specialised\":" << (K.specialised ? "true" : "false");
    }
    o << ",\"bytes\":" << K.bytes << ",\"m\":" << K.m << ",\"n\":" << K.n << ",\"bind\":[";
    for (size_t j = 0; j < K.bind.size(); ++j)
      o << (j ? "," : "") << "[\"" << field_name(K, (size_t)(uintptr_t)K.bind[j].first) << "\"," << K.bind[j].second << "]";
    o << "]}";
  }
  o << "]}";
  const std::string str = o.str();
  if (needed) *needed = str.size() + 1;
  if (buf != nullptr && cap > 0) {
    const size_t k = std::min(cap - 1, str.size());
    std::memcpy(buf, str.data(), k);
    buf[k] = 0;
  }
  return KF_OK;
}

kf_status kf_plan_execute(const kf_plan* p, void* const* bindings, int n_bindings, void* ws, size_t ws_bytes,
                          void* stream) {
  if (p == nullptr || (n_bindings > 0 && bindings == nullptr)) return err(KF_ERR_INVALID_ARG, "null argument");
  if (n_bindings < p->nvars) return err(KF_ERR_INVALID_ARG, "every script variable needs a binding");
  kf_status chk = check_plan(p->p, bindings, n_bindings, ws, ws_bytes);
  if (chk != KF_OK) return chk;
  const MatTune tune = current_matrix_tuning();
  for (const Kernel& K : p->p.kernels) {
    kf_status st = launch_kernel(K, bindings, n_bindings, ws, ws_bytes, stream, tune);
    if (st != KF_OK) return st;
  }
  return KF_OK;
}

kf_status kf_plan_time(const kf_plan* p, void* const* bindings, int n_bindings, void* ws, size_t ws_bytes,
                       void* stream, int reps, float* median_ms) {
  if (p == nullptr || median_ms == nullptr || reps <= 0) return err(KF_ERR_INVALID_ARG, "bad arguments");
  return time_plan(p->p, p->nvars, bindings, n_bindings, ws, ws_bytes, stream, reps, median_ms);
}

kf_status kf_planner_set_model(double bw_gbs, double launch_us) {
  if (bw_gbs <= 0 || launch_us < 0) return err(KF_ERR_INVALID_ARG, "bandwidth must be positive");
  set_model(bw_gbs * 1e9, launch_us);
  return KF_OK;
}


kf_status kf_autotune_plan(const kf_plan* p, void* const* bindings, int n_bindings, void* ws, size_t ws_bytes,
                           void* stream, int reps, float* tuned_ms, float* auto_ms) {
  if (p == nullptr || reps <= 0 || (n_bindings > 0 && bindings == nullptr)) return err(KF_ERR_INVALID_ARG, "bad arguments");
  if (n_bindings < p->nvars) return err(KF_ERR_INVALID_ARG, "every script variable needs a binding");
  kf_status chk = check_plan(p->p, bindings, n_bindings, ws, ws_bytes);
  if (chk != KF_OK) return chk;
  float tsum = 0.f, asum = 0.f;
  for (const Kernel& K : p->p.kernels) {
    float bm = 0.f, am = 0.f;
    if (K.is_atax) continue;  // tuned on first use by its own search (ring depth, blocks per SM, clusters)
    if (K.is_mat) {
      MatProg P = K.mp;
      for (auto& b : K.bind) {
        if (b.second < 0 || b.second >= n_bindings || bindings[b.second] == nullptr)
          return err(KF_ERR_INVALID_ARG, "variable " + std::to_string(b.second) + " is not bound");
        *reinterpret_cast<void**>(reinterpret_cast<char*>(&P) + (size_t)(uintptr_t)b.first) = bindings[b.second];
      }
      char* wsm = ws ? static_cast<char*>(ws) + plan_vec_region() : nullptr;
      const size_t wsm_bytes = ws_bytes > plan_vec_region() ? ws_bytes - plan_vec_region() : 0;
      if ((P.nrow_res || P.ncol_res || P.nrow_out || P.ncol_out) && matprog_bind_workspace(P, wsm, wsm_bytes) != 0)
        return err(KF_ERR_WORKSPACE, "workspace missing or smaller than kf_plan_workspace_size()");
      MatTune best{};
      const int rc = autotune_matprog(P, stream, reps, &best, &bm, &am);
      if (rc != 0) return err(rc, "autotune failed");
    } else {
      VecProg P = K.vp;
      for (auto& b : K.bind) {
        if (b.second < 0 || b.second >= n_bindings || bindings[b.second] == nullptr)
          return err(KF_ERR_INVALID_ARG, "variable " + std::to_string(b.second) + " is not bound");
        *reinterpret_cast<void**>(reinterpret_cast<char*>(&P) + (size_t)(uintptr_t)b.first) = bindings[b.second];
      }
      if (P.ndot > 0) {
        if (ws == nullptr || ws_bytes < plan_vec_region()) return err(KF_ERR_WORKSPACE, "workspace too small");
        P.counter = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + WS_HEADER);
        P.dotpart = reinterpret_cast<float*>(static_cast<char*>(ws) + WS_HEADER + 256);
      }
      P.fp64_final = P.n >= (int64_t(1) << 26);
      VecTune best{};
      const int rc = autotune_vecprog(P, stream, reps, &best, &bm, &am);
      if (rc != 0) return err(rc, "autotune failed");
    }
    tsum += bm;
    asum += am;
  }
  if (tuned_ms) *tuned_ms = tsum;
  if (auto_ms) *auto_ms = asum;
  return KF_OK;
}

kf_status kf_tune_cache_clear(void) {
  tune_cache_clear();
  return KF_OK;
}

kf_status kf_tune_cache_entries(int* n) {
  if (n == nullptr) return err(KF_ERR_INVALID_ARG, "null argument");
  *n = (int)tune_cache_size();
  return KF_OK;
}

static std::string device_tag() {
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return "unknown";
  std::string name = prop.name;
  for (char& c : name)
    if (c == ' ') c = '_';
  return name + "_sm" + std::to_string(prop.multiProcessorCount);
}

kf_status kf_tune_cache_save(const char* path) {
  if (path == nullptr) return err(KF_ERR_INVALID_ARG, "null path");
  std::vector<std::string> lines;
  tune_cache_dump(&lines);
  std::ofstream f(path);
  if (!f) return err(KF_ERR_INVALID_ARG, std::string("cannot write ") + path);
  f << "# kf tuning cache v1\ndevice " << device_tag() << "\n";
  for (auto& l : lines) f << l << "\n";
  return f ? KF_OK : err(KF_ERR_INVALID_ARG, "write failed");
}

kf_status kf_tune_cache_load(const char* path, int* loaded) {
  if (path == nullptr) return err(KF_ERR_INVALID_ARG, "null path");
  std::ifstream f(path);
  if (!f) return err(KF_ERR_INVALID_ARG, std::string("cannot read ") + path);
  std::string line;
  int n = 0;
  bool dev_ok = false;
  while (std::getline(f, line)) {
    if (line.empty() || line[0] == '#') continue;
    if (line.rfind("device ", 0) == 0) {
      dev_ok = line.substr(7) == device_tag();
      continue;
    }
    if (!dev_ok) continue;  // tunings of another device are not used
    const size_t colon = line.find(" : ");
    if (colon == std::string::npos) return err(KF_ERR_INVALID_ARG, "malformed tuning cache line: " + line);
    const std::string key = line.substr(0, colon);
    int v[5] = {0, 0, 0, 0, 0};
    const int got = std::sscanf(line.c_str() + colon + 3, "%d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4]);
    if ((key.rfind("mat ", 0) == 0 || key.rfind("atax ", 0) == 0 || key.rfind("gemver_form ", 0) == 0 ||
         key.rfind("sgemvt_form ", 0) == 0) &&
        got == 5) {
      tune_cache_put_mat(key, MatTune{v[0], v[1], v[2], v[3], v[4]});
      ++n;
    } else if (key.rfind("vec ", 0) == 0 && got == 3) {
      tune_cache_put_vec(key, VecTune{v[0], v[1], v[2]});
      ++n;
    } else {
      return err(KF_ERR_INVALID_ARG, "malformed tuning cache line: " + line);
    }
  }
  if (loaded) *loaded = n;
  return KF_OK;
}


// Features, analytic prediction and kernel count of every enumerated plan
// (index order of KF_PLAN_INDEX), in one call.
kf_status kf_plan_enumerate_info(const kf_script* s, int cap, float* feats, double* pred_us, int* kernels,
                                 int* count) {
  if (s == nullptr || count == nullptr || cap <= 0) return err(KF_ERR_INVALID_ARG, "bad arguments");
  kf_status st = ensure_analysed(s);
  if (st != KF_OK) return st;
  std::vector<std::vector<std::vector<int>>> all;
  bool tr = false;
  enumerate(s->s, (size_t)cap, &all, &tr);
  std::vector<float> f;
  for (size_t i = 0; i < all.size(); ++i) {
    Plan p;
    std::string e = make_plan(s->s, all[i], &p);
    if (!e.empty()) return err(KF_ERR_UNSUPPORTED, e);
    if (feats) {
      features(s->s, p, &f);
      std::copy(f.begin(), f.end(), feats + i * NFEATURES);
    }
    if (pred_us) pred_us[i] = p.predicted_us;
    if (kernels) kernels[i] = (int)p.kernels.size();
  }
  *count = (int)all.size();
  return KF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Plan selection: analytic ranking, learned ranking pruning the empirical
// search, exhaustive empirical search (Section 3.2).
namespace {

constexpr int SELECT_DEFAULT_CAP = 2000;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct Enumerated {
  std::vector<Plan> plans;
  size_t ws_max = 0;  // largest plan workspace
};

kf_status enumerate_built(const kf_script* s, int cap, Enumerated* E) {
  kf_status st = ensure_analysed(s);
  if (st != KF_OK) return st;
  std::vector<std::vector<std::vector<int>>> all;
  bool tr = false;
  enumerate(s->s, (size_t)cap, &all, &tr);
  if (all.empty()) return err(KF_ERR_UNSUPPORTED, "no legal plan");
  E->plans.resize(all.size());
  for (size_t i = 0; i < all.size(); ++i) {
    std::string e = make_plan(s->s, all[i], &E->plans[i]);
    if (!e.empty()) return err(KF_ERR_UNSUPPORTED, e);
    E->ws_max = std::max(E->ws_max, E->plans[i].ws_bytes);
  }
  return KF_OK;
}

// [plans' region | standardised features (count x 16) | predictions (count)]
size_t select_ws_bytes(const Enumerated& E) {
  const size_t n = E.plans.size();
  return align256(E.ws_max) + align256(n * NFEATURES * sizeof(float)) + align256(n * sizeof(float));
}

kf_status check_bindings(const kf_script* s, void* const* bindings, int nb) {
  if (bindings == nullptr) return err(KF_ERR_INVALID_ARG, "timing needs bindings");
  if (nb < (int)s->s.vars.size()) return err(KF_ERR_INVALID_ARG, "every script variable needs a binding");
  return KF_OK;
}

}  // namespace

extern "C" {

kf_status kf_plan_select_workspace_size(const kf_script* s, int max_plans, size_t* bytes) {
  if (s == nullptr || bytes == nullptr) return err(KF_ERR_INVALID_ARG, "null argument");
  Enumerated E;
  kf_status st = enumerate_built(s, max_plans > 0 ? max_plans : SELECT_DEFAULT_CAP, &E);
  if (st != KF_OK) return st;
  *bytes = select_ws_bytes(E);
  return KF_OK;
}

kf_status kf_plan_time_all(const kf_script* s, int max_plans, void* const* bindings, int n_bindings, void* ws,
                           size_t ws_bytes, void* stream, int reps, float* ms, int* count) {
  if (s == nullptr || ms == nullptr || count == nullptr) return err(KF_ERR_INVALID_ARG, "null argument");
  Enumerated E;
  kf_status st = enumerate_built(s, max_plans > 0 ? max_plans : SELECT_DEFAULT_CAP, &E);
  if (st != KF_OK) return st;
  if ((st = check_bindings(s, bindings, n_bindings)) != KF_OK) return st;
  if (ws_bytes < select_ws_bytes(E) || (ws == nullptr && E.ws_max > 0))
    return err(KF_ERR_WORKSPACE, "workspace smaller than kf_plan_select_workspace_size()");
  const int nvars = (int)s->s.vars.size();
  for (size_t i = 0; i < E.plans.size(); ++i) {
    st = time_plan(E.plans[i], nvars, bindings, n_bindings, ws, ws_bytes, stream, reps > 0 ? reps : 3, &ms[i]);
    if (st != KF_OK) return st;
  }
  *count = (int)E.plans.size();
  return KF_OK;
}

kf_status kf_plan_select(const kf_script* s, const kf_select_options* opt, const kf_cost_model* model,
                         void* const* bindings, int n_bindings, void* ws, size_t ws_bytes, void* stream, kf_plan** out,
                         kf_select_info* info) {
  if (s == nullptr || opt == nullptr || out == nullptr) return err(KF_ERR_INVALID_ARG, "null argument");
  const int cap = opt->max_plans > 0 ? opt->max_plans : SELECT_DEFAULT_CAP;
  const int reps = opt->reps > 0 ? opt->reps : 3;
  Enumerated E;
  kf_status st = enumerate_built(s, cap, &E);
  if (st != KF_OK) return st;
  const int count = (int)E.plans.size();
  const int nvars = (int)s->s.vars.size();
  cudaStream_t cs = (cudaStream_t)stream;
  int chosen = 0;
  double predicted = 0.0;
  std::vector<int> cand;  // plans to time
  if (opt->mode == KF_SELECT_ANALYTIC) {
    for (int i = 1; i < count; ++i)
      if (E.plans[i].predicted_us < E.plans[chosen].predicted_us * (1.0 - 1e-9)) chosen = i;
    predicted = E.plans[chosen].predicted_us;
  } else if (opt->mode == KF_SELECT_MLP) {
    if (model == nullptr || model->params == nullptr) return err(KF_ERR_INVALID_ARG, "KF_SELECT_MLP needs a model");
    if (ws == nullptr || ws_bytes < select_ws_bytes(E))
      return err(KF_ERR_WORKSPACE, "workspace smaller than kf_plan_select_workspace_size()");
    std::vector<float> X((size_t)count * NFEATURES), f;
    for (int i = 0; i < count; ++i) {
      features(s->s, E.plans[i], &f);
      for (int c = 0; c < NFEATURES; ++c)
        X[(size_t)i * NFEATURES + c] = (f[c] - model->mean[c]) * model->inv_std[c];
    }
    float* dX = reinterpret_cast<float*>(static_cast<char*>(ws) + align256(E.ws_max));
    float* dY = reinterpret_cast<float*>(reinterpret_cast<char*>(dX) + align256(X.size() * sizeof(float)));
    std::vector<float> y(count);
    if (cudaMemcpyAsync(dX, X.data(), X.size() * sizeof(float), cudaMemcpyHostToDevice, cs) != cudaSuccess)
      return err(KF_ERR_CUDA, "copy of plan features failed");
    st = kf_mlp_forward(model->params, NFEATURES, 64, dX, count, dY, stream);
    if (st != KF_OK) return st;
    if (cudaMemcpyAsync(y.data(), dY, count * sizeof(float), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess)
      return err(KF_ERR_CUDA, "cost model evaluation failed");
    if (model->analytic_weight != 0.f)
      for (int i = 0; i < count; ++i)
        y[i] += model->analytic_weight * (float)std::log(std::max(E.plans[i].predicted_us, 1e-3) * 1e-3);
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return y[a] < y[b]; });
    chosen = order[0];
    predicted = y[chosen];
    // the top_k best-ranked plans, plus (margin > 0) every plan scored within
    // `margin` of the best, at most 64: ambiguous rankings are settled by timing
    int ntime = opt->top_k > 1 ? std::min(opt->top_k, count) : 0;
    if (opt->margin > 0.f) {
      int nm = 0;
      while (nm < count && nm < 64 && y[order[nm]] - y[order[0]] <= opt->margin) ++nm;
      if (nm > 1) ntime = std::max(ntime, nm);
    }
    if (ntime > 1) cand.assign(order.begin(), order.begin() + ntime);
  } else if (opt->mode == KF_SELECT_EXHAUSTIVE) {
    cand.resize(count);
    for (int i = 0; i < count; ++i) cand[i] = i;
  } else {
    return err(KF_ERR_INVALID_ARG, "unknown selection mode");
  }
  float best_ms = 0.f;
  if (!cand.empty()) {
    if ((st = check_bindings(s, bindings, n_bindings)) != KF_OK) return st;
    if (ws_bytes < select_ws_bytes(E) || (ws == nullptr && E.ws_max > 0))
      return err(KF_ERR_WORKSPACE, "workspace smaller than kf_plan_select_workspace_size()");
    best_ms = 3.4e38f;
    for (int i : cand) {
      float ms = 0.f;
      st = time_plan(E.plans[i], nvars, bindings, n_bindings, ws, ws_bytes, stream, reps, &ms);
      if (st != KF_OK) return st;
      if (ms < best_ms) {
        best_ms = ms;
        chosen = i;
      }
    }
    if (opt->mode == KF_SELECT_EXHAUSTIVE) predicted = E.plans[chosen].predicted_us;
  }
  auto* pl = new (std::nothrow) kf_plan();
  if (pl == nullptr) return err(KF_ERR_NO_MEM, "out of host memory");
  pl->p = std::move(E.plans[chosen]);
  pl->nvars = nvars;
  *out = pl;
  if (info) {
    info->index = chosen;
    info->count = count;
    info->timed = (int)cand.size();
    info->best_ms = best_ms;
    info->predicted = predicted;
  }
  return KF_OK;
}

}  // extern "C"
