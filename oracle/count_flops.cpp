// count_flops.cpp -- counting instantiation of the oracle (TEST INFRASTRUCTURE ONLY).
//
// Compiles oracle.c with REAL = Counted, a number type that records every
// arithmetic operation as a node of an expression graph, and counts the
// algorithmic work of the volume term (Section 4.1) from the oracle's own
// code:
//   * per unordered node pair: the oracle's volume_pair() for both orderings
//     (i, l) and (l, i), with common subexpressions shared -- the two-point
//     flux, its log means and the metric average are symmetric and evaluated
//     once, the gravity term and the accumulation into each node twice, which
//     is the work of the half sweep over pairs;
//   * per node: primitives() once, volume_value() for the five values and one
//     lsrk_value() stage update for each.
// Conventions: +, -, *, / (and sqrt, log) count one flop each; negation and
// comparisons count none; an operation whose operands are all compile-time
// constants (literals, the LGL operator) or run-time parameters (gamma, the
// step and stage coefficients) is hoisted and counts none; shared
// subexpressions are found by hash-consing with commutative operands sorted
// and signs moved outward (b - a is -(a - b), (-x)(-y) is x y), so an operand
// order or sign convention of the oracle changes no count.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <tuple>
#include <type_traits>
#include <vector>

namespace flopcount {

enum Kind { CONSTANT = 0, PARAM = 1, DATA = 2 };
enum Op { LEAF = 0, ADD = 1, MUL = 2, DIV = 3, SQRT = 4, LOG = 5, ABS = 6 };

struct Node {
  int op, a, b, kind;  // operands as signed references (see Ref)
};

// A reference is node id * 2 + sign bit (1 = negated).
struct Graph {
  std::vector<Node> nodes;
  std::map<std::tuple<int, int, int>, int> cons;  // (op, a, b) -> node id
  std::map<std::pair<int, double>, int> leaves;   // constants by value
  int leaf(int kind, double value, bool unique) {
    if (!unique) {
      auto it = leaves.find({kind, value});
      if (it != leaves.end()) return it->second * 2;
    }
    nodes.push_back(Node{LEAF, 0, 0, kind});
    const int id = (int)nodes.size() - 1;
    if (!unique) leaves[{kind, value}] = id;
    return id * 2;
  }
  int kind(int ref) const { return nodes[ref >> 1].kind; }
  // returns a reference to op(a, b) with canonical operands; sign of the result
  // is folded into the returned reference
  int make(int op, int a, int b) {
    int sign = 0;
    if (op == ADD) {
      if (b >> 1 < a >> 1) std::swap(a, b);
      if (a & 1) {  // (-a) + b -> -(a + (-b))
        a ^= 1;
        b ^= 1;
        sign = 1;
      }
    } else if (op == MUL || op == DIV) {
      sign = (a & 1) ^ (b & 1);
      a &= ~1;
      b &= ~1;
      if (op == MUL && b < a) std::swap(a, b);
    } else if (op == SQRT || op == LOG) {
      b = 0;
    } else if (op == ABS) {
      a &= ~1;
      b = 0;
    }
    const int k = std::max(kind(a), op == ADD || op == MUL || op == DIV ? kind(b) : 0);
    auto key = std::make_tuple(op, a, b);
    auto it = cons.find(key);
    int id;
    if (it != cons.end()) {
      id = it->second;
    } else {
      nodes.push_back(Node{op, a, b, k});
      id = (int)nodes.size() - 1;
      cons[key] = id;
    }
    return id * 2 + sign;
  }
  // data-dependent operations reachable from the given references
  long long count(const std::vector<int>& outs) const {
    std::vector<char> seen(nodes.size(), 0);
    std::vector<int> stack;
    for (int r : outs) stack.push_back(r >> 1);
    long long n = 0;
    while (!stack.empty()) {
      const int id = stack.back();
      stack.pop_back();
      if (seen[id]) continue;
      seen[id] = 1;
      const Node& nd = nodes[id];
      if (nd.op == LEAF) continue;
      if (nd.kind == DATA) n++;
      stack.push_back(nd.a >> 1);
      if (nd.op == ADD || nd.op == MUL || nd.op == DIV) stack.push_back(nd.b >> 1);
    }
    return n;
  }
};

Graph* G = nullptr;
bool make_params = false;  // conversions from floating values create run-time parameters

}  // namespace flopcount

// The counted number type: a value (for the oracle's branch decisions) and a
// graph reference.  Eight bytes, like double, so sizeof-based choices in the
// oracle take their double branch.
struct Counted {
  float v;
  int32_t r;
  Counted() : v(0.0f), r(flopcount::G->leaf(flopcount::CONSTANT, 0.0, false)) {}
  Counted(int x) : v((float)x), r(flopcount::G->leaf(flopcount::CONSTANT, (double)x, false)) {}
  Counted(double x)
      : v((float)x),
        r(flopcount::G->leaf(flopcount::make_params ? flopcount::PARAM : flopcount::CONSTANT, x,
                             false)) {}
  Counted(long double x) : Counted((double)x) {}
  static Counted data(double x) {
    Counted c;
    c.v = (float)x;
    c.r = flopcount::G->leaf(flopcount::DATA, x, true);
    return c;
  }
  static Counted param(double x) {
    Counted c;
    c.v = (float)x;
    c.r = flopcount::G->leaf(flopcount::PARAM, x, true);
    return c;
  }
  explicit operator double() const { return v; }
  explicit operator long double() const { return v; }
  explicit operator float() const { return v; }
};
static_assert(sizeof(Counted) == sizeof(double), "the oracle's double branch");

inline Counted mk(float v, int r) {
  Counted c;
  c.v = v;
  c.r = r;
  return c;
}
inline Counted operator-(Counted a) { return mk(-a.v, a.r ^ 1); }
inline Counted operator+(Counted a, Counted b) {
  return mk(a.v + b.v, flopcount::G->make(flopcount::ADD, a.r, b.r));
}
inline Counted operator-(Counted a, Counted b) {
  return mk(a.v - b.v, flopcount::G->make(flopcount::ADD, a.r, b.r ^ 1));
}
inline Counted operator*(Counted a, Counted b) {
  return mk(a.v * b.v, flopcount::G->make(flopcount::MUL, a.r, b.r));
}
inline Counted operator/(Counted a, Counted b) {
  return mk(a.v / b.v, flopcount::G->make(flopcount::DIV, a.r, b.r));
}
inline Counted& operator+=(Counted& a, Counted b) { return a = a + b; }
inline Counted& operator-=(Counted& a, Counted b) { return a = a - b; }
inline Counted& operator*=(Counted& a, Counted b) { return a = a * b; }
inline Counted& operator/=(Counted& a, Counted b) { return a = a / b; }
#define COUNTED_MIXED(OP)                                                        \
  template <typename T, typename = typename std::enable_if<std::is_arithmetic<T>::value>::type> \
  inline Counted operator OP(Counted a, T b) { return a OP Counted(b); }        \
  template <typename T, typename = typename std::enable_if<std::is_arithmetic<T>::value>::type> \
  inline Counted operator OP(T a, Counted b) { return Counted(a) OP b; }
COUNTED_MIXED(+)
COUNTED_MIXED(-)
COUNTED_MIXED(*)
COUNTED_MIXED(/)
inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { return a.v >= b.v; }
inline bool operator==(Counted a, Counted b) { return a.v == b.v; }
inline bool operator!=(Counted a, Counted b) { return a.v != b.v; }
inline Counted sqrt(Counted a) { return mk(std::sqrt(a.v), flopcount::G->make(flopcount::SQRT, a.r, 0)); }
inline Counted log(Counted a) { return mk(std::log(a.v), flopcount::G->make(flopcount::LOG, a.r, 0)); }
inline Counted fabs(Counted a) { return mk(std::fabs(a.v), flopcount::G->make(flopcount::ABS, a.r, 0)); }
// functions of the oracle's initial states (not on the counted paths)
inline Counted exp(Counted a) { return mk(std::exp(a.v), flopcount::G->make(flopcount::LOG, a.r ^ 1, 0)); }
inline Counted cos(Counted a) { return mk(std::cos(a.v), flopcount::G->make(flopcount::SQRT, a.r ^ 1, 0)); }
inline Counted tanh(Counted a) { return mk(std::tanh(a.v), flopcount::G->make(flopcount::ABS, a.r, 0)); }
inline Counted pow(Counted a, Counted b) { return exp(b * log(a)); }

#define REAL Counted
#include "oracle.c"

namespace {
using flopcount::G;

prim_t data_prim(double rho, double u0, double u1, double u2, double p, double phi) {
  prim_t s;
  s.rho = Counted::data(rho);
  s.u[0] = Counted::data(u0);
  s.u[1] = Counted::data(u1);
  s.u[2] = Counted::data(u2);
  s.p = Counted::data(p);
  s.b = Counted::data(rho / (2.0 * p));
  s.phi = Counted::data(phi);
  return s;
}
}  // namespace

// Counts for order N (1..7): out[0] flops per unordered node pair of the half
// sweep, out[1] flops per node and stage (primitives, the five volume values
// and their stage updates), out[2] primitives, out[3] one stage update of one
// value, out[4] the pair's two orderings without sharing.  Returns 0, or -1
// for an unsupported order.
extern "C" int or_count_flops(int N, double* out) {
  flopcount::Graph graph;
  G = &graph;
  basis_t B;
  if (N < 1 || N > 7 || build_basis(N, &B)) {
    G = nullptr;
    return -1;
  }
  const Counted gamma = Counted::param(1.4);
  // a pair of nodes along direction 0 at indices a = 0, m = 1 of a one-element
  // pencil; states close to each other (the log means' series branch, the
  // branch the workloads take)
  const int np = (N + 1) * (N + 1) * (N + 1);
  std::vector<Counted> Ja(9 * np);
  for (int k = 0; k < 9 * np; k++) Ja[k] = Counted::data(1.0 + 0.01 * k);
  const prim_t Pi = data_prim(1.16, 0.3, -0.2, 0.1, 9.9e4, 4.9e3);
  const prim_t Pl = data_prim(1.161, 0.31, -0.21, 0.12, 9.91e4, 4.91e3);
  const int i = node_with(&B, 0, 0, 0), l = node_with(&B, 0, 0, 1);
  Counted acc_i[NV], acc_l[NV], acc_i2[NV], acc_l2[NV];
  for (int v = 0; v < NV; v++) {
    acc_i[v] = Counted::data(0.1 * v);
    acc_l[v] = Counted::data(0.2 * v);
  }
  std::memcpy(acc_i2, acc_i, sizeof(acc_i));
  std::memcpy(acc_l2, acc_l, sizeof(acc_l));
  volume_pair(&B, Ja.data(), np, 0, i, l, 0, 1, &Pi, &Pl, gamma, acc_i);
  volume_pair(&B, Ja.data(), np, 0, l, i, 1, 0, &Pl, &Pi, gamma, acc_l);
  std::vector<int> outs;
  for (int v = 0; v < NV; v++) {
    outs.push_back(acc_i[v].r);
    outs.push_back(acc_l[v].r);
  }
  const long long pair_shared = graph.count(outs);
  // without sharing: each ordering in a graph of its own
  long long pair_separate = 0;
  for (int o = 0; o < 2; o++) {
    flopcount::Graph g2;
    G = &g2;
    basis_t B2;
    build_basis(N, &B2);
    const Counted gm = Counted::param(1.4);
    std::vector<Counted> Ja2(9 * np);
    for (int k = 0; k < 9 * np; k++) Ja2[k] = Counted::data(1.0 + 0.01 * k);
    const prim_t A2 = data_prim(1.16, 0.3, -0.2, 0.1, 9.9e4, 4.9e3);
    const prim_t C2 = data_prim(1.161, 0.31, -0.21, 0.12, 9.91e4, 4.91e3);
    Counted acc[NV];
    for (int v = 0; v < NV; v++) acc[v] = Counted::data(0.1 * v);
    if (o == 0) volume_pair(&B2, Ja2.data(), np, 0, i, l, 0, 1, &A2, &C2, gm, acc);
    else volume_pair(&B2, Ja2.data(), np, 0, l, i, 1, 0, &C2, &A2, gm, acc);
    std::vector<int> o2;
    for (int v = 0; v < NV; v++) o2.push_back(acc[v].r);
    pair_separate += g2.count(o2);
  }
  G = &graph;
  // per node: primitives from the conserved state
  Counted q[NV];
  q[0] = Counted::data(1.16);
  q[1] = Counted::data(0.35);
  q[2] = Counted::data(-0.23);
  q[3] = Counted::data(0.12);
  q[4] = Counted::data(2.5e5);
  const prim_t pn = primitives(q, Counted::data(4.9e3), gamma);
  const long long prims = graph.count({pn.u[0].r, pn.u[1].r, pn.u[2].r, pn.p.r, pn.b.r});
  // per value: the volume value and one stage update (a stage after the first:
  // the register holds data)
  const Counted vv = volume_value(Counted::data(3.0), Counted::data(0.5));
  Counted dq = Counted::data(0.01), qv = Counted::data(1.16);
  lsrk_value(vv, Counted::data(0.2), Counted::data(0.0), Counted::param(-0.4),
             Counted::param(0.37), Counted::param(0.03), &dq, &qv);
  const long long value = graph.count({dq.r, qv.r});
  const long long stage = value - graph.count({vv.r});
  out[0] = (double)pair_shared;
  out[1] = (double)(prims + NV * value);
  out[2] = (double)prims;
  out[3] = (double)stage;
  out[4] = (double)pair_separate;
  G = nullptr;
  return 0;
}
