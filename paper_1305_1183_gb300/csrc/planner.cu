// Script analysis, fusion legality, plan enumeration and kernel composition.
// (Host code.  See planner.h for the scheme.)
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <set>

#include "planner.h"

namespace kf {
namespace plan {

namespace {

bool is_vec(const Script& s, int v) { return s.vars[v].kind == VK_VECTOR; }
bool is_mat(const Script& s, int v) { return s.vars[v].kind == VK_MATRIX; }
int64_t vlen(const Script& s, int v) { return s.vars[v].n; }

// Which input positions of a call are vector operands indexed by matrix rows
// (length m) or columns (length n) for matrix ops.
// GEMV: x (col), y0 (row); GEMVT: y (row), x0 (col); GER: u (row), v (col).
int vec_side(int op, int pos) {  // 0 row, 1 col, -1 n/a
  if (op == OP_GEMV) return pos == 1 ? 1 : (pos == 2 ? 0 : -1);
  if (op == OP_GEMVT) return pos == 1 ? 0 : (pos == 2 ? 1 : -1);
  if (op == OP_GER) return pos == 1 ? 0 : (pos == 2 ? 1 : -1);
  return -1;
}

}  // namespace

std::string analyse(Script& s) {
  const int nv = (int)s.vars.size(), nc = (int)s.calls.size();
  std::vector<int> cur(nv, 0);
  s.writer.assign(nv, std::vector<int>(1, -1));
  s.readers.assign(nv, std::vector<std::vector<int>>(1));
  for (int c = 0; c < nc; ++c) {
    Call& k = s.calls[c];
    auto need = [&](bool ok, const char* msg) -> std::string { return ok ? "" : std::string(msg); };
    std::string e;
    const size_t ni = k.ins.size();
    if (k.outs.size() != 1) return "every call has exactly one output";
    for (int v : k.ins)
      if (v < 0 || v >= nv) return "input variable id out of range";
    if (k.outs[0] < 0 || k.outs[0] >= nv) return "output variable id out of range";
    const int o = k.outs[0];
    switch (k.op) {
      case OP_AXPBY:
        e = need(ni == 2 && is_vec(s, k.ins[0]) && is_vec(s, k.ins[1]) && is_vec(s, o) &&
                     vlen(s, k.ins[0]) == vlen(s, o) && vlen(s, k.ins[1]) == vlen(s, o),
                 "AXPBY: out = a x + b y over vectors of one length");
        break;
      case OP_SCAL:
        e = need(ni == 1 && is_vec(s, k.ins[0]) && is_vec(s, o) && vlen(s, k.ins[0]) == vlen(s, o),
                 "SCAL: out = a x over vectors of one length");
        break;
      case OP_VADD:
        e = need(ni == 3 && is_vec(s, k.ins[0]) && is_vec(s, k.ins[1]) && is_vec(s, k.ins[2]) && is_vec(s, o) &&
                     vlen(s, k.ins[0]) == vlen(s, o) && vlen(s, k.ins[1]) == vlen(s, o) &&
                     vlen(s, k.ins[2]) == vlen(s, o),
                 "VADD: out = w + y + z over vectors of one length");
        break;
      case OP_DOT:
        e = need(ni == 2 && is_vec(s, k.ins[0]) && is_vec(s, k.ins[1]) && s.vars[o].kind == VK_SCALAR &&
                     vlen(s, k.ins[0]) == vlen(s, k.ins[1]),
                 "DOT: scalar = x . y over vectors of one length");
        break;
      case OP_GEMV:
        e = need((ni == 2 || ni == 3) && is_mat(s, k.ins[0]) && is_vec(s, k.ins[1]) && is_vec(s, o) &&
                     vlen(s, k.ins[1]) == s.vars[k.ins[0]].n && vlen(s, o) == s.vars[k.ins[0]].m &&
                     (ni == 2 || (is_vec(s, k.ins[2]) && vlen(s, k.ins[2]) == s.vars[k.ins[0]].m)) &&
                     o != k.ins[1],
                 "GEMV: y = a A x + b y0 (A m x n, x length n, y and y0 length m, y not x)");
        break;
      case OP_GEMVT:
        e = need((ni == 2 || ni == 3) && is_mat(s, k.ins[0]) && is_vec(s, k.ins[1]) && is_vec(s, o) &&
                     vlen(s, k.ins[1]) == s.vars[k.ins[0]].m && vlen(s, o) == s.vars[k.ins[0]].n &&
                     (ni == 2 || (is_vec(s, k.ins[2]) && vlen(s, k.ins[2]) == s.vars[k.ins[0]].n)) &&
                     o != k.ins[1],
                 "GEMVT: x = a A^T y + b x0 (A m x n, y length m, x and x0 length n, x not y)");
        break;
      case OP_GER:
        e = need(ni == 3 && is_mat(s, k.ins[0]) && is_vec(s, k.ins[1]) && is_vec(s, k.ins[2]) && is_mat(s, o) &&
                     vlen(s, k.ins[1]) == s.vars[k.ins[0]].m && vlen(s, k.ins[2]) == s.vars[k.ins[0]].n &&
                     s.vars[o].m == s.vars[k.ins[0]].m && s.vars[o].n == s.vars[k.ins[0]].n,
                 "GER: B = A + a u v^T (u length m, v length n, B the shape of A)");
        break;
      default: return "unknown op";
    }
    if (!e.empty()) return e;
    k.depth = (k.op == OP_GEMV || k.op == OP_GEMVT || k.op == OP_GER) ? 2 : 1;
    k.in_ver.resize(ni);
    for (size_t i = 0; i < ni; ++i) {
      const int v = k.ins[i];
      if (cur[v] == 0 && !s.vars[v].input) return "variable '" + s.vars[v].name + "' is read before it is written";
      k.in_ver[i] = cur[v];
      s.readers[v][cur[v]].push_back(c);
    }
    cur[o]++;
    k.out_ver = cur[o];
    s.writer[o].push_back(c);
    s.readers[o].emplace_back();
  }
  s.final_ver = cur;
  // dependency graph
  s.succ.assign(nc, {});
  s.pred.assign(nc, {});
  auto edge = [&](int a, int b) {
    if (a < 0 || a == b) return;
    if (std::find(s.succ[a].begin(), s.succ[a].end(), b) == s.succ[a].end()) {
      s.succ[a].push_back(b);
      s.pred[b].push_back(a);
    }
  };
  for (int c = 0; c < nc; ++c) {
    const Call& k = s.calls[c];
    for (size_t i = 0; i < k.ins.size(); ++i) edge(s.writer[k.ins[i]][k.in_ver[i]], c);   // RAW
    const int o = k.outs[0];
    for (int r : s.readers[o][k.out_ver - 1]) edge(r, c);                                // WAR
    edge(s.writer[o][k.out_ver - 1], c);                                                  // WAW
  }
  s.reach.assign(nc, std::vector<char>(nc, 0));
  for (int c = nc - 1; c >= 0; --c)
    for (int d : s.succ[c]) {
      s.reach[c][d] = 1;
      for (int e2 = 0; e2 < nc; ++e2)
        if (s.reach[d][e2]) s.reach[c][e2] = 1;
    }
  s.analysed = true;
  return "";
}

namespace {

struct Val {  // a variable version
  int var, ver;
  bool operator<(const Val& o) const { return var != o.var ? var < o.var : ver < o.ver; }
  bool operator==(const Val& o) const { return var == o.var && ver == o.ver; }
};

bool in_group(const std::vector<int>& g, int c) { return std::find(g.begin(), g.end(), c) != g.end(); }

// Is (var, ver) produced by a call of g?
bool produced_in(const Script& s, const std::vector<int>& g, int var, int ver) {
  const int w = s.writer[var][ver];
  return w >= 0 && in_group(g, w);
}

// Is (var, ver), produced in g, needed after g?  `placed` limits the test to
// calls already assigned (partial plans), or all calls when null.
bool live_out(const Script& s, const std::vector<int>& g, int var, int ver, const std::vector<char>* placed) {
  if (s.vars[var].output && ver == s.final_ver[var]) return true;
  for (int r : s.readers[var][ver])
    if (!in_group(g, r) && (placed == nullptr || (*placed)[r])) return true;
  // the final version of a non-output variable read by nobody is dead
  return false;
}

// Symbolic linear expression: term -> coefficient.
using Expr = std::map<std::pair<int, int>, double>;  // (kind 0 raw-row 1 raw-col 2 ext-var, id)

void add_scaled(Expr& dst, const Expr& src, double a) {
  for (auto& kv : src) dst[kv.first] += a * kv.second;
}

}  // namespace

// Single-pass ATAX: {t = a1 A x; y = a2 A^T t} over one version of A, with t
// needed by nothing else and no accumulated terms.  The row dot t_i is a
// reduction consumed in the same kernel, which the fusion rules otherwise
// forbid (a global barrier is needed); a block that owns whole rows (the
// persistent row reuse Section 4.2 names) finishes t_i before it uses it, so
// the pair runs with one read of A when a row fits the shared-memory ring.
bool atax_pair(const Script& s, const std::vector<int>& g0, const std::vector<char>* placed) {
  if (g0.size() != 2) return false;
  std::vector<int> g = g0;
  std::sort(g.begin(), g.end());
  const Call& a = s.calls[g[0]];
  const Call& b = s.calls[g[1]];
  if (a.op != OP_GEMV || b.op != OP_GEMVT) return false;
  if (a.ins[0] != b.ins[0] || a.in_ver[0] != b.in_ver[0]) return false;
  if (b.ins[1] != a.outs[0] || b.in_ver[1] != a.out_ver) return false;
  if ((a.ins.size() > 2 && a.sc[1] != 0.0) || (b.ins.size() > 2 && b.sc[1] != 0.0)) return false;
  if (live_out(s, g, a.outs[0], a.out_ver, placed)) return false;
  const Var& A = s.vars[a.ins[0]];
  return A.m >= 1 && A.n >= 4 && A.n % 4 == 0 && A.n <= 16384;
}

bool legal_group_impl(const Script& s, const std::vector<int>& g, std::string* why,
                      const std::vector<char>* placed) {
  auto fail = [&](const char* m) { if (why) *why = m; return false; };
  if (g.empty()) return fail("empty");
  // convexity: no path leaving and re-entering the group
  const int nc = (int)s.calls.size();
  for (int a : g)
    for (int b : g)
      if (a != b && s.reach[a][b])
        for (int x = a + 1; x < b; ++x)
          if (!in_group(g, x) && s.reach[a][x] && s.reach[x][b]) return fail("not convex");
  (void)nc;
  int maxdepth = 0;
  for (int c : g) maxdepth = std::max(maxdepth, s.calls[c].depth);
  // no two live versions of one variable written in the group
  std::map<int, int> live_versions;
  for (int c : g) {
    const Call& k = s.calls[c];
    if (live_out(s, g, k.outs[0], k.out_ver, placed)) live_versions[k.outs[0]]++;
  }
  for (auto& kv : live_versions)
    if (kv.second > 1) return fail("two versions of one variable are needed after the fusion");

  if (maxdepth == 1) {
    // ---- vector pass: one length, limits on inputs / outputs / dots
    int64_t len = -1;
    std::set<int> ext_in;
    int nout = 0, ndot = 0;
    for (int c : g) {
      const Call& k = s.calls[c];
      for (size_t i = 0; i < k.ins.size(); ++i) {
        const int v = k.ins[i];
        if (len < 0) len = vlen(s, v);
        if (vlen(s, v) != len) return fail("vectors of different lengths");
        if (!produced_in(s, g, v, k.in_ver[i])) ext_in.insert(v);
      }
      if (k.op == OP_DOT) ++ndot;
      else {
        if (vlen(s, k.outs[0]) != len) return fail("vectors of different lengths");
        if (live_out(s, g, k.outs[0], k.out_ver, placed)) ++nout;
      }
    }
    if ((int)ext_in.size() > VP_MAXIN) return fail("too many input vectors");
    if (nout > VP_MAXOUT) return fail("too many output vectors");
    if (ndot > VP_MAXDOT) return fail("too many dot products");
    return true;
  }

  if (atax_pair(s, g, placed)) return true;

  // ---- matrix pass (depth-2 core) with optional linear epilogue maps
  int64_t m = -1, n = -1;
  int nops = 0, ngemv = 0;
  struct Lineage { Val cur; };
  std::vector<Lineage> lin;
  std::map<Val, int> row_res, col_res;  // reduction results produced in g -> side
  std::set<int> row_written, col_written, row_read_ext, col_read_ext;
  std::map<Val, int> epi_side;          // epilogue values produced in g -> side
  for (int c : g) {
    const Call& k = s.calls[c];
    if (k.depth == 2) {
      const int A = k.ins[0];
      if (m < 0) { m = s.vars[A].m; n = s.vars[A].n; }
      if (s.vars[A].m != m || s.vars[A].n != n) return fail("matrices of different shapes");
      ++nops;
      // matrix operand: an entry version or the current version of a lineage
      const Val av{A, k.in_ver[0]};
      int li = -1;
      for (size_t q = 0; q < lin.size(); ++q)
        if (lin[q].cur == av) li = (int)q;
      if (li < 0) {
        if (produced_in(s, g, A, k.in_ver[0])) return fail("an older version of a matrix updated in the fusion");
        lin.push_back({av});
        li = (int)lin.size() - 1;
      }
      // vector operands must come from outside the fusion
      for (size_t i = 1; i < k.ins.size(); ++i) {
        if (produced_in(s, g, k.ins[i], k.in_ver[i])) return fail("a reduction result consumed in the fusion");
        if (vec_side(k.op, (int)i) == 0) row_read_ext.insert(k.ins[i]);
        else col_read_ext.insert(k.ins[i]);
      }
      if (k.op == OP_GER) lin[li].cur = Val{k.outs[0], k.out_ver};
      else if (k.op == OP_GEMV) { ++ngemv; row_res[Val{k.outs[0], k.out_ver}] = 0; row_written.insert(k.outs[0]); }
      else { col_res[Val{k.outs[0], k.out_ver}] = 1; col_written.insert(k.outs[0]); }
    } else {
      // epilogue map: reads at least one reduction (or epilogue) value of g
      if (k.op == OP_DOT) return fail("a dot product of a reduction result needs another barrier");
      int side = -1;
      for (size_t i = 0; i < k.ins.size(); ++i) {
        const Val v{k.ins[i], k.in_ver[i]};
        int sd = -1;
        if (row_res.count(v)) sd = 0;
        else if (col_res.count(v)) sd = 1;
        else if (epi_side.count(v)) sd = epi_side[v];
        else if (produced_in(s, g, v.var, v.ver)) return fail("map of a value the epilogue cannot see");
        if (sd >= 0) {
          if (side >= 0 && side != sd) return fail("epilogue mixes row and column results");
          side = sd;
        }
      }
      if (side < 0) return fail("a map that reads no reduction result of the matrix pass");
      for (size_t i = 0; i < k.ins.size(); ++i) {
        const Val v{k.ins[i], k.in_ver[i]};
        if (!row_res.count(v) && !col_res.count(v) && !epi_side.count(v)) {
          if (side == 0) row_read_ext.insert(v.var); else col_read_ext.insert(v.var);
        }
      }
      epi_side[Val{k.outs[0], k.out_ver}] = side;
      if (side == 0) row_written.insert(k.outs[0]); else col_written.insert(k.outs[0]);
    }
  }
  if (nops == 0) return fail("no matrix op");
  if (nops > MAT_MAXOPS) return fail("too many matrix ops");
  if (ngemv > 2) return fail("more than two GEMV results");
  if (lin.size() > 2) return fail("more than two matrices");
  // A row-indexed write must not meet a column-indexed read of the same
  // vector (or the reverse): other blocks may still be reading it.
  for (int v : row_written) if (col_read_ext.count(v)) return fail("row result aliases a column operand");
  for (int v : col_written) if (row_read_ext.count(v)) return fail("column result aliases a row operand");
  // Matrix intermediates: only a lineage's last version may be needed later.
  for (int c : g) {
    const Call& k = s.calls[c];
    if (k.op != OP_GER) continue;
    const Val out{k.outs[0], k.out_ver};
    bool is_cur = false;
    for (auto& l : lin) is_cur = is_cur || l.cur == out;
    if (!is_cur && live_out(s, g, out.var, out.ver, placed)) return fail("an intermediate matrix is needed later");
  }
  // epilogue outputs per side
  int nrow_out = 0, ncol_out = 0;
  for (int c : g) {
    const Call& k = s.calls[c];
    const Val out{k.outs[0], k.out_ver};
    if (k.op == OP_GER) continue;
    if (!live_out(s, g, out.var, out.ver, placed)) continue;
    int side = row_res.count(out) ? 0 : col_res.count(out) ? 1 : epi_side.count(out) ? epi_side[out] : -1;
    if (side == 0) ++nrow_out; else if (side == 1) ++ncol_out;
  }
  if (nrow_out > EPI_MAXOUT || ncol_out > EPI_MAXOUT) return fail("too many epilogue outputs");
  return true;
}

bool legal_group(const Script& s, const std::vector<int>& g, std::string* why) {
  return legal_group_impl(s, g, why, nullptr);
}

namespace {

bool quotient_order(const Script& s, const std::vector<std::vector<int>>& groups, std::vector<int>* order) {
  const int nc = (int)s.calls.size();
  std::vector<int> gid(nc, -1);
  for (size_t i = 0; i < groups.size(); ++i)
    for (int c : groups[i]) gid[c] = (int)i;
  const int ng = (int)groups.size();
  std::vector<std::set<int>> gsucc(ng);
  std::vector<int> indeg(ng, 0);
  for (int c = 0; c < nc; ++c)
    for (int d : s.succ[c])
      if (gid[c] != gid[d] && gsucc[gid[c]].insert(gid[d]).second) indeg[gid[d]]++;
  // Kahn's algorithm; ties by the earliest call of the group
  std::vector<int> ready;
  for (int i = 0; i < ng; ++i)
    if (indeg[i] == 0) ready.push_back(i);
  order->clear();
  while (!ready.empty()) {
    std::sort(ready.begin(), ready.end(), [&](int a, int b) { return groups[a][0] > groups[b][0]; });
    const int x = ready.back();
    ready.pop_back();
    order->push_back(x);
    for (int y : gsucc[x])
      if (--indeg[y] == 0) ready.push_back(y);
  }
  return (int)order->size() == ng;
}

}  // namespace

void enumerate(const Script& s, size_t cap, std::vector<std::vector<std::vector<int>>>* out, bool* truncated) {
  const int nc = (int)s.calls.size();
  out->clear();
  *truncated = false;
  std::vector<std::vector<int>> groups;
  std::vector<char> placed(nc, 0);
  std::vector<int> order;
  std::function<void(int)> rec = [&](int i) {
    if (*truncated) return;
    if (i == nc) {
      for (auto& g : groups)
        if (!legal_group_impl(s, g, nullptr, nullptr)) return;
      if (!quotient_order(s, groups, &order)) return;
      if (out->size() >= cap) { *truncated = true; return; }  // a plan beyond the cap exists
      out->push_back(groups);
      return;
    }
    placed[i] = 1;
    for (size_t gi = 0; gi < groups.size() && !*truncated; ++gi) {
      groups[gi].push_back(i);
      if (legal_group_impl(s, groups[gi], nullptr, &placed)) rec(i + 1);
      groups[gi].pop_back();
    }
    if (!*truncated) {
      groups.push_back({i});
      if (legal_group_impl(s, groups.back(), nullptr, &placed)) rec(i + 1);
      groups.pop_back();
    }
    placed[i] = 0;
  };
  rec(0);
}

// ---------------------------------------------------------------- composition

namespace {

// Analytic model (the paper's predictor, Section 3.2, sums transfer time t_t
// and compute time t_c of a fusion separately and predicts max(t_t, t_c)):
// t_t = bytes moved / g_bw, t_c = flops / g_flops, plus a fixed cost per
// kernel, which the paper's predictor leaves out (Section 4.3 names that
// omission as the cause of its AXPYDOT misprediction).  For these
// memory-bound calls t_c is far below t_t.
double g_bw = 6.5e12;        // bytes/s
double g_flops = 80e12;      // FP32 FMA rate of the GPU (152 SMs x 128 lanes x 2 x 2.07 GHz)
double g_launch_us = 2.0;    // fixed cost per kernel

// Floating-point operations of one call (2 per multiply-add).
double call_flops(const Script& s, const Call& c) {
  const Var& o = s.vars[c.outs.empty() ? c.ins[0] : c.outs[0]];
  switch (c.op) {
    case OP_GEMV:
    case OP_GEMVT:
    case OP_GER: {
      const Var& A = s.vars[c.ins[0]];
      return 2.0 * (double)A.m * (double)A.n;
    }
    case OP_DOT: return 2.0 * (double)s.vars[c.ins[0]].n;
    case OP_SCAL: return (double)o.n;
    default: return 3.0 * (double)o.n;  // AXPBY, VADD
  }
}

template <typename T>
size_t off(const T& base, const void* field) {
  return (size_t)(static_cast<const char*>(field) - reinterpret_cast<const char*>(&base));
}

}  // namespace

void set_model(double bw_bytes_per_s, double launch_us) {
  if (bw_bytes_per_s > 0) g_bw = bw_bytes_per_s;
  if (launch_us >= 0) g_launch_us = launch_us;
}
void get_model(double* bw, double* launch_us) {
  *bw = g_bw;
  *launch_us = g_launch_us;
}

static std::string build_vec_kernel(const Script& s, const std::vector<int>& g, Kernel* K) {
  VecProg& P = K->vp;
  std::memset(&P, 0, sizeof(P));
  std::vector<int> inputs;  // external input variables (entry versions)
  std::map<Val, std::vector<double>> coef;
  auto input_index = [&](int v) {
    for (size_t i = 0; i < inputs.size(); ++i)
      if (inputs[i] == v) return (int)i;
    inputs.push_back(v);
    return (int)inputs.size() - 1;
  };
  // first pass: collect inputs in order of first use
  for (int c : g) {
    const Call& k = s.calls[c];
    for (size_t i = 0; i < k.ins.size(); ++i)
      if (!produced_in(s, g, k.ins[i], k.in_ver[i])) input_index(k.ins[i]);
  }
  if ((int)inputs.size() > VP_MAXIN) return "too many inputs";
  const int NI = (int)inputs.size();
  auto expr = [&](int v, int ver) -> std::vector<double> {
    auto it = coef.find(Val{v, ver});
    if (it != coef.end()) return it->second;
    std::vector<double> e(NI, 0.0);
    e[input_index(v)] = 1.0;
    return e;
  };
  int64_t len = 0;
  for (int c : g) {
    const Call& k = s.calls[c];
    len = vlen(s, k.ins[0]);
    std::vector<double> r(NI, 0.0);
    auto acc = [&](int i, double a) {
      auto e = expr(k.ins[i], k.in_ver[i]);
      for (int q = 0; q < NI; ++q) r[q] += a * e[q];
    };
    switch (k.op) {
      case OP_AXPBY: acc(0, k.sc[0]); if (k.sc[1] != 0.0) acc(1, k.sc[1]); break;
      case OP_SCAL: acc(0, k.sc[0]); break;
      case OP_VADD: acc(0, 1.0); acc(1, 1.0); acc(2, 1.0); break;
      case OP_DOT: {
        if (P.ndot >= VP_MAXDOT) return "too many dots";
        auto a = expr(k.ins[0], k.in_ver[0]);
        auto b = expr(k.ins[1], k.in_ver[1]);
        for (int q = 0; q < NI; ++q) { P.P[P.ndot][q] = (float)a[q]; P.Q[P.ndot][q] = (float)b[q]; }
        K->bind.push_back({(void**)(uintptr_t)off(P, &P.dot_out[P.ndot]), k.outs[0]});
        P.ndot++;
        continue;
      }
      default: return "not a vector op";
    }
    coef[Val{k.outs[0], k.out_ver}] = r;
  }
  for (int c : g) {
    const Call& k = s.calls[c];
    if (k.op == OP_DOT) continue;
    if (!live_out(s, g, k.outs[0], k.out_ver, nullptr)) continue;
    if (P.nout >= VP_MAXOUT) return "too many outputs";
    auto r = coef[Val{k.outs[0], k.out_ver}];
    for (int q = 0; q < NI; ++q) P.C[P.nout][q] = (float)r[q];
    K->bind.push_back({(void**)(uintptr_t)off(P, &P.out[P.nout]), k.outs[0]});
    P.nout++;
  }
  P.nin = NI;
  for (int i = 0; i < NI; ++i) K->bind.push_back({(void**)(uintptr_t)off(P, &P.in[i]), inputs[i]});
  P.n = len;
  K->n = len;
  K->bytes = 4.0 * (double)len * (NI + P.nout) + 4.0 * P.ndot;
  return "";
}

// Call-order search (Section 3.2, fusion variant (i): the order of the
// calls inside a fusion).  Two matrix calls of a fusion keep their script
// order when one writes a variable the other reads or writes; a GER
// rewrites the row values in place, so the calls reading the version it
// replaces go first even though the script's versions do not depend on
// each other.  Any other pair may swap, and every order that keeps these
// pairs computes the same bits for every result (each result is its own
// sum in its own fixed order).  The order decides the op signature, and
// with it whether a specialised kernel instance exists: the search takes
// the script order if it has one, else the first legal permutation in
// lexicographic order that has one, else the script order.  The linear
// epilogue maps, which only read the matrix calls' results, follow the
// matrix calls in script order.
static std::vector<int> search_call_order(const Script& s, const std::vector<int>& g, bool* specialised) {
  std::vector<int> M, E;
  for (int c : g) (s.calls[c].depth == 2 ? M : E).push_back(c);
  auto touches = [&](int c, int v) {
    const Call& k = s.calls[c];
    if (k.outs[0] == v) return true;
    for (int i : k.ins)
      if (i == v) return true;
    return false;
  };
  auto conflict = [&](int a, int b) { return touches(b, s.calls[a].outs[0]) || touches(a, s.calls[b].outs[0]); };
  // kinds and matrix slots of an order, slots by first appearance of each
  // matrix lineage (a GER's output continues its input's lineage)
  auto compiled = [&](const std::vector<int>& order) {
    std::vector<std::pair<int, int>> lin;
    int kinds[8], mats[8], nops = 0;
    for (int c : order) {
      const Call& k = s.calls[c];
      const std::pair<int, int> av{k.ins[0], k.in_ver[0]};
      int li = -1;
      for (size_t q = 0; q < lin.size(); ++q)
        if (lin[q] == av) li = (int)q;
      if (li < 0) {
        lin.push_back(av);
        li = (int)lin.size() - 1;
      }
      if (nops >= 8) return false;
      kinds[nops] = k.op == OP_GER ? MOP_GER : (k.op == OP_GEMV ? MOP_GEMV : MOP_GEMVT);
      mats[nops] = li;
      ++nops;
      if (k.op == OP_GER) lin[li] = {k.outs[0], k.out_ver};
    }
    return matprog_sig_compiled(kinds, mats, nops, FMT_F32);
  };
  *specialised = compiled(M);
  std::vector<int> out = g;
  if (*specialised || M.size() < 2 || M.size() > 6) return out;
  // an epilogue result read by a matrix call pins the script order
  for (int e : E)
    for (int c : M)
      if (touches(c, s.calls[e].outs[0])) return out;
  std::vector<int> perm(M.size());
  for (size_t i = 0; i < perm.size(); ++i) perm[i] = (int)i;
  while (std::next_permutation(perm.begin(), perm.end())) {
    bool legal = true;
    for (size_t i = 0; i < perm.size() && legal; ++i)
      for (size_t j = i + 1; j < perm.size() && legal; ++j)
        if (perm[i] > perm[j] && conflict(M[perm[i]], M[perm[j]])) legal = false;
    if (!legal) continue;
    std::vector<int> order;
    for (int i : perm) order.push_back(M[i]);
    if (compiled(order)) {
      *specialised = true;
      out = order;
      out.insert(out.end(), E.begin(), E.end());
      return out;
    }
  }
  return out;
}

static std::string build_mat_kernel(const Script& s, const std::vector<int>& g, Kernel* K) {
  MatProg& P = K->mp;
  std::memset(&P, 0, sizeof(P));
  struct Lin { Val cur; int slot; int entry_var; };
  std::vector<Lin> lin;
  std::map<Val, Expr> vexpr;         // row/col values produced in g
  std::map<Val, int> side;           // 0 row 1 col
  std::set<int> ext_vectors;         // distinct external vectors read (bytes)
  bool specialised = false;
  const std::vector<int> order = search_call_order(s, g, &specialised);
  K->order = order;
  K->specialised = specialised;
  for (int c : order) {
    const Call& k = s.calls[c];
    if (k.depth == 2) {
      const int A = k.ins[0];
      P.m = s.vars[A].m;
      P.n = s.vars[A].n;
      const Val av{A, k.in_ver[0]};
      int li = -1;
      for (size_t q = 0; q < lin.size(); ++q)
        if (lin[q].cur == av) li = (int)q;
      if (li < 0) {
        lin.push_back({av, (int)lin.size(), A});
        li = (int)lin.size() - 1;
        P.fmt = FMT_F32;
        K->bind.push_back({(void**)(uintptr_t)off(P, &P.A[li]), A});
        P.lda[li] = s.vars[A].ld;
      }
      MatOp& op = P.ops[P.nops];
      op.mat = lin[li].slot;
      if (k.op == OP_GER) {
        op.kind = MOP_GER;
        op.alpha = (float)k.sc[0];
        K->bind.push_back({(void**)(uintptr_t)off(P, &op.rowvec), k.ins[1]});
        K->bind.push_back({(void**)(uintptr_t)off(P, &op.colvec), k.ins[2]});
        ext_vectors.insert(k.ins[1]);
        ext_vectors.insert(k.ins[2]);
        lin[li].cur = Val{k.outs[0], k.out_ver};
      } else if (k.op == OP_GEMV) {
        op.kind = MOP_GEMV;
        op.res = P.nrow_res++;
        K->bind.push_back({(void**)(uintptr_t)off(P, &op.colvec), k.ins[1]});
        ext_vectors.insert(k.ins[1]);
        Expr e;
        e[{0, op.res}] = k.sc[0];
        if (k.ins.size() > 2 && k.sc[1] != 0.0) { e[{2, k.ins[2]}] += k.sc[1]; ext_vectors.insert(k.ins[2]); }
        vexpr[Val{k.outs[0], k.out_ver}] = e;
        side[Val{k.outs[0], k.out_ver}] = 0;
      } else {
        op.kind = MOP_GEMVT;
        op.res = P.ncol_res++;
        K->bind.push_back({(void**)(uintptr_t)off(P, &op.rowvec), k.ins[1]});
        ext_vectors.insert(k.ins[1]);
        Expr e;
        e[{1, op.res}] = k.sc[0];
        if (k.ins.size() > 2 && k.sc[1] != 0.0) { e[{2, k.ins[2]}] += k.sc[1]; ext_vectors.insert(k.ins[2]); }
        vexpr[Val{k.outs[0], k.out_ver}] = e;
        side[Val{k.outs[0], k.out_ver}] = 1;
      }
      P.nops++;
    } else {
      // epilogue map
      Expr e;
      int sd = -1;
      auto acc = [&](int i, double a) {
        const Val v{k.ins[i], k.in_ver[i]};
        auto it = vexpr.find(v);
        if (it != vexpr.end()) { add_scaled(e, it->second, a); sd = side[v]; }
        else { e[{2, v.var}] += a; ext_vectors.insert(v.var); }
      };
      switch (k.op) {
        case OP_AXPBY: acc(0, k.sc[0]); if (k.sc[1] != 0.0) acc(1, k.sc[1]); break;
        case OP_SCAL: acc(0, k.sc[0]); break;
        case OP_VADD: acc(0, 1.0); acc(1, 1.0); acc(2, 1.0); break;
        default: return "not an epilogue op";
      }
      vexpr[Val{k.outs[0], k.out_ver}] = e;
      side[Val{k.outs[0], k.out_ver}] = sd;
    }
  }
  P.nmat = (int)lin.size();
  // stored matrices: the last version of each lineage, when a GER of the
  // fusion produced it and it is needed after the fusion
  double mat_bytes = 0.0;
  for (auto& l : lin) {
    mat_bytes += 4.0 * (double)P.m * (double)P.n;
    if (produced_in(s, g, l.cur.var, l.cur.ver) && live_out(s, g, l.cur.var, l.cur.ver, nullptr)) {
      K->bind.push_back({(void**)(uintptr_t)off(P, &P.Bout[l.slot]), l.cur.var});
      P.ldb[l.slot] = s.vars[l.cur.var].ld;
      mat_bytes += 4.0 * (double)P.m * (double)P.n;
    }
  }
  // epilogue outputs
  double vec_bytes = 0.0;
  for (int c : order) {
    const Call& k = s.calls[c];
    if (k.op == OP_GER) continue;
    const Val out{k.outs[0], k.out_ver};
    if (!live_out(s, g, out.var, out.ver, nullptr)) continue;
    const int sd = side[out];
    EpiOut& o = (sd == 0) ? P.row_out[P.nrow_out] : P.col_out[P.ncol_out];
    const int idx = (sd == 0) ? P.nrow_out : P.ncol_out;
    std::memset(&o, 0, sizeof(o));
    for (auto& kv : vexpr[out]) {
      if (kv.second == 0.0) continue;
      if (o.nterm >= EPI_MAXTERM) return "epilogue expression too long";
      if (kv.first.first == 2) {
        o.src[o.nterm] = -1;
        K->bind.push_back({(void**)(uintptr_t)off(P, &o.ext[o.nterm]), kv.first.second});
      } else {
        o.src[o.nterm] = kv.first.second;
      }
      o.coef[o.nterm] = (float)kv.second;
      o.nterm++;
    }
    if (o.nterm == 0) { o.src[0] = -1; o.coef[0] = 0.f; }  // identically zero: write zeros
    K->bind.push_back({(void**)(uintptr_t)off(P, &o.dst), out.var});
    vec_bytes += 4.0 * (double)vlen(s, out.var);
    if (sd == 0) P.nrow_out++; else P.ncol_out++;
    (void)idx;
  }
  for (int v : ext_vectors) vec_bytes += 4.0 * (double)vlen(s, v);
  K->m = P.m;
  K->n = P.n;
  K->bytes = mat_bytes + vec_bytes;
  K->is_mat = true;
  return "";
}

static std::string build_atax_kernel(const Script& s, const std::vector<int>& g0, Kernel* K) {
  std::vector<int> g = g0;
  std::sort(g.begin(), g.end());
  const Call& a = s.calls[g[0]];
  const Call& b = s.calls[g[1]];
  const int A = a.ins[0];
  K->is_atax = true;
  K->atax_scale = (float)(a.sc[0] * b.sc[0]);
  K->bind.push_back({(void**)(uintptr_t)0, A});
  K->bind.push_back({(void**)(uintptr_t)1, a.ins[1]});
  K->bind.push_back({(void**)(uintptr_t)2, b.outs[0]});
  K->m = s.vars[A].m;
  K->n = s.vars[A].n;
  K->lda = s.vars[A].ld;
  K->bytes = 4.0 * (double)K->m * (double)K->n + 8.0 * (double)K->n;  // A once, x in, y out
  return "";
}

std::string make_plan(const Script& s, const std::vector<std::vector<int>>& groups, Plan* p) {
  p->groups = groups;
  for (auto& g : p->groups) std::sort(g.begin(), g.end());
  if (!quotient_order(s, p->groups, &p->order)) return "the fusions cannot be ordered (cycle)";
  p->kernels.clear();
  p->predicted_us = 0.0;
  p->bytes = 0.0;
  // workspace: a region for vector passes, then one for matrix passes
  const size_t vec_region = (vecprog_workspace_bytes(VP_MAXDOT) + 255) & ~(size_t)255;
  p->ws_bytes = vec_region;
  for (int gi : p->order) {
    const auto& g = p->groups[gi];
    std::string why;
    if (!legal_group(s, g, &why)) return "illegal fusion: " + why;
    Kernel K;
    K.calls = g;
    int depth = 1;
    for (int c : g) depth = std::max(depth, s.calls[c].depth);
    K.depth = depth;
    std::string e = depth == 2 ? (atax_pair(s, g, nullptr) ? build_atax_kernel(s, g, &K) : build_mat_kernel(s, g, &K))
                               : build_vec_kernel(s, g, &K);
    if (!e.empty()) return e;
    if (K.is_atax) {
      p->ws_bytes = std::max(p->ws_bytes, vec_region + atax_plan_workspace_bytes(K.m, K.n));
    } else if (K.is_mat) {
      const size_t w = matprog_workspace_bytes(K.mp.m, K.mp.n, std::max(K.mp.nrow_res, 1), std::max(K.mp.ncol_res, 1), FMT_F32);
      p->ws_bytes = std::max(p->ws_bytes, vec_region + w);
    } else {
      p->ws_bytes = std::max(p->ws_bytes, vec_region);
    }
    p->bytes += K.bytes;
    double flops = 0.0;
    for (int c : g) flops += call_flops(s, s.calls[c]);
    p->predicted_us += std::max(K.bytes / g_bw, flops / g_flops) * 1e6 + g_launch_us;
    p->kernels.push_back(std::move(K));
  }
  return "";
}

void features(const Script& s, const Plan& p, std::vector<float>* f) {
  f->assign(NFEATURES, 0.f);
  float nk = (float)p.kernels.size(), nmat = 0, nvec = 0, maxops = 0;
  double matb = 0, vecb = 0, minb = 1e300;
  float rowfin = 0, colfin = 0, dotk = 0, nepi = 0, nstore = 0;
  int64_t nmax = 1;
  for (const auto& K : p.kernels) {
    minb = std::min(minb, K.bytes);
    if (K.is_atax) {
      // one matrix pass (two matrix calls) whose column results need a second phase
      nmat += 1;
      matb += 4.0 * K.m * K.n;
      vecb += K.bytes - 4.0 * K.m * K.n;
      maxops = std::max(maxops, 2.f);
      colfin += 1;
      nepi += 1;
      nmax = std::max<int64_t>(nmax, std::max(K.m, K.n));
    } else if (K.is_mat) {
      nmat += 1;
      matb += 4.0 * K.m * K.n * K.mp.nmat;
      vecb += K.bytes - 4.0 * K.m * K.n * K.mp.nmat;
      maxops = std::max(maxops, (float)K.mp.nops);
      rowfin += K.mp.nrow_res > 0;  // a second, dependent phase for row results
      colfin += K.mp.ncol_res > 0;  // ... and for column results
      nepi += (float)(K.mp.nrow_out + K.mp.ncol_out);
      nmax = std::max<int64_t>(nmax, std::max(K.m, K.n));
    } else {
      nvec += 1;
      vecb += K.bytes;
      dotk += K.vp.ndot > 0;
      nmax = std::max<int64_t>(nmax, K.n);
    }
  }
  for (const auto& K : p.kernels)
    for (const auto& b : K.bind)
      for (int t = 0; t < 2; ++t)
        if (K.is_mat && (size_t)(uintptr_t)b.first == off(K.mp, &K.mp.Bout[t])) nstore += 1;
  // byte counts span orders of magnitude across sizes: log scale
  (*f)[0] = nk;
  (*f)[1] = nmat;
  (*f)[2] = nvec;
  (*f)[3] = (float)std::log2(1.0 + p.bytes);
  (*f)[4] = (float)std::log2(1.0 + matb);
  (*f)[5] = (float)std::log2(1.0 + vecb);
  (*f)[6] = (float)std::log2((double)nmax);
  (*f)[7] = nk > 0 ? (float)s.calls.size() / nk : 0.f;
  (*f)[8] = maxops;
  (*f)[9] = rowfin;
  (*f)[10] = colfin;
  (*f)[11] = dotk;
  (*f)[12] = (float)std::log2(1.0 + (nk > 0 ? minb : 0.0));
  (*f)[13] = (float)std::log2(1.0 + p.predicted_us);
  (*f)[14] = nepi;
  (*f)[15] = nstore;
}

}  // namespace plan
}  // namespace kf
