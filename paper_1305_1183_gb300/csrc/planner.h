// Script, dependency graph, fusion plans (host side of libkf).
//
// The paper's compiler (Section 3.2) turns a script of elementary calls into
// a data-dependency graph, generates the fusible subgraphs ("fusions"),
// implementations of each and combinations that cover every call, ranks
// them with a performance predictor and optionally searches them
// empirically.  Here:
//   * every write of a variable creates a new version (the script's order
//     and data dependencies define the result, Section 3.1); edges are
//     read-after-write, write-after-read and write-after-write;
//   * a fusion is a set of calls of the same nesting depth over the same
//     iteration space (map/reduce fusion rules of Section 3.2.1-3.2.3), in
//     which no reduction result is consumed, except by linear maps that run
//     after the last-block barrier (the epilogue), convex in the graph;
//   * a plan is a partition of the calls into fusions whose quotient graph
//     is acyclic; plans are enumerated call by call in script order;
//   * a fusion becomes one launch of the vector-pass or matrix-pass kernel
//     (kf_internal.h), composed from its calls.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "kf_internal.h"

namespace kf {
namespace plan {

enum VarKind { VK_VECTOR = 0, VK_MATRIX = 1, VK_SCALAR = 2 };

// Op codes (kf.h kf_op).
enum Op { OP_AXPBY = 0, OP_SCAL = 1, OP_DOT = 2, OP_VADD = 3, OP_GEMV = 4, OP_GEMVT = 5, OP_GER = 6 };

struct Var {
  std::string name;
  int kind;
  int64_t m, n;  // vector: n; matrix: m x n; scalar: 1
  int64_t ld = 0;  // matrix: row stride in elements (>= n; n unless declared)
  bool input = false, output = false;
};

struct Call {
  int op;
  std::vector<int> outs, ins;
  double sc[2] = {0.0, 0.0};
  // filled by analyse()
  std::vector<int> in_ver;   // version of each input read
  int out_ver = 0;           // version written
  int depth = 1;             // 1: vectors, 2: matrices
};

struct Script {
  std::vector<Var> vars;
  std::vector<Call> calls;
  // analysis
  bool analysed = false;
  std::vector<int> final_ver;                       // per variable
  std::vector<std::vector<int>> writer;             // [var][version] -> call or -1
  std::vector<std::vector<std::vector<int>>> readers;  // [var][version] -> calls
  std::vector<std::vector<int>> succ, pred;         // dependency graph over calls
  std::vector<std::vector<char>> reach;             // transitive closure
};

// Kernel produced for one fusion.
struct Kernel {
  std::vector<int> calls;  // in script order
  std::vector<int> order;  // matrix pass: the calls in kernel order (call-order search)
  bool specialised = false;  // matrix pass: a specialised instance exists for that order
  int depth = 1;
  bool is_mat = false;
  // Single-pass ATAX, y = atax_scale * A^T (A x): bind holds A, x, y in that
  // order (their offsets are 0, 1, 2); it runs as kf_atax's kernels.
  bool is_atax = false;
  float atax_scale = 1.f;
  MatProg mp{};            // pointers hold var ids (cast) until bound
  VecProg vp{};
  // binding maps: for each pointer field, which variable it refers to
  std::vector<std::pair<void**, int>> bind;  // filled per execution on a copy
  double bytes = 0.0;      // bytes moved (model)
  int64_t m = 0, n = 0;
  int64_t lda = 0;         // single-pass ATAX: row stride of A
};

struct Plan {
  std::vector<std::vector<int>> groups;  // calls per fusion
  std::vector<int> order;                // schedule (indices into groups)
  std::vector<Kernel> kernels;           // in schedule order
  double predicted_us = 0.0;             // analytic model
  double bytes = 0.0;
  size_t ws_bytes = 0;
};

// Returns an empty string on success, else the reason.
std::string analyse(Script& s);
// Is the set of calls a legal fusion?  (reason in *why when not)
bool legal_group(const Script& s, const std::vector<int>& g, std::string* why);
// Enumerate plans (up to cap); each plan is a partition with acyclic quotient.
void enumerate(const Script& s, size_t cap, std::vector<std::vector<std::vector<int>>>* out, bool* truncated);
// Build kernels and the analytic prediction for a partition.
std::string make_plan(const Script& s, const std::vector<std::vector<int>>& groups, Plan* p);
// Feature vector of a plan for the learned cost model.
void features(const Script& s, const Plan& p, std::vector<float>* f);
constexpr int NFEATURES = 16;

}  // namespace plan
}  // namespace kf
