// Algorithmic operation counts of the DG-HGKS point computations.
//
// The device flux functions of gks_point.cuh are instantiated on the host
// with a counting scalar: every distinct +, -, *, / between two values is one
// floating-point operation (value numbering removes repeated subexpressions
// and operations with constant 0 or +-1 operands), and sqrt, exp, erfc are
// counted apart (they run on the special-function pipe and as
// multi-instruction sequences).  The
// trace evaluation (modal -> Gauss point values and gradients) and the
// quadrature projections are counted from their loop structure, keeping
// only terms whose basis factor is not identically zero.
//
// Output (stdout): one JSON object per (order, n_q, Pr != 1) with the counts
// per face point and per cell point.  The benchmark divides the counted
// operations of one launch by its measured duration for the roofline.
#define DG_HD inline
#include <cmath>
#include <cstdio>
#include <map>
#include <set>
#include <tuple>
#include <utility>
#include <vector>

namespace opc {
// Value numbering: every distinct (operation, operands) pair is counted once,
// as a compiler's common-subexpression elimination would; operations with a
// compile-time constant 0 or +-1 operand are free (folded).  The point inputs
// and gas parameters are run-time values with ids of their own.
struct Tally {
  long add = 0, mul = 0, div = 0, sqrt = 0, exp = 0, erfc = 0;
  long flops() const { return add + mul + div; }
};
Tally g;
std::map<std::tuple<char, int, int>, int> memo;
std::map<int, std::tuple<char, int, int>> nodes;  // the operation that produced each id
std::map<double, int> const_ids;
std::map<int, double> const_vals;
int next_id = 1;

inline int const_id(double x) {
  auto it = const_ids.find(x);
  if (it != const_ids.end()) return it->second;
  const int id = next_id++;
  const_ids[x] = id;
  const_vals[id] = x;
  return id;
}
inline bool is_const(int id, double x) {
  auto it = const_vals.find(id);
  return it != const_vals.end() && it->second == x;
}
inline void reset() {
  g = Tally();
  memo.clear();
  nodes.clear();
}

struct Cnt {
  double v;
  int id;
  Cnt() : v(0), id(const_id(0.0)) {}
  Cnt(double x) : v(x), id(const_id(x)) {}
  Cnt(double x, int i) : v(x), id(i) {}
};

// returns the id of (op, a, b), counting it in *slot if it is new
inline int vn(char op, int a, int b, long* slot) {
  if (op == '+' || op == '*')
    if (a > b) std::swap(a, b);
  auto key = std::make_tuple(op, a, b);
  auto it = memo.find(key);
  if (it != memo.end()) return it->second;
  if (slot) ++*slot;
  const int id = next_id++;
  memo[key] = id;
  nodes[id] = key;
  return id;
}

// Operations on which the given results depend (what remains after a
// compiler removes the code whose results are never used).
inline Tally live(const std::vector<int>& outs) {
  Tally t;
  std::set<int> seen;
  std::vector<int> stack(outs.begin(), outs.end());
  while (!stack.empty()) {
    const int id = stack.back();
    stack.pop_back();
    if (!seen.insert(id).second) continue;
    auto it = nodes.find(id);
    if (it == nodes.end()) continue;  // constant or input
    const char op = std::get<0>(it->second);
    if (op == '+' || op == '-') ++t.add;
    else if (op == '*') ++t.mul;
    else if (op == '/') ++t.div;
    else if (op == 's') ++t.sqrt;
    else if (op == 'e') ++t.exp;
    else if (op == 'c') ++t.erfc;
    stack.push_back(std::get<1>(it->second));
    if (op != 'n' && op != 's' && op != 'e' && op != 'c') stack.push_back(std::get<2>(it->second));
  }
  return t;
}
inline Cnt operator+(Cnt a, Cnt b) {
  if (is_const(a.id, 0.0)) return b;
  if (is_const(b.id, 0.0)) return a;
  return Cnt(a.v + b.v, vn('+', a.id, b.id, &g.add));
}
inline Cnt operator-(Cnt a, Cnt b) {
  if (is_const(b.id, 0.0)) return a;
  return Cnt(a.v - b.v, vn('-', a.id, b.id, &g.add));
}
inline Cnt operator*(Cnt a, Cnt b) {
  if (is_const(a.id, 0.0) || is_const(b.id, 0.0)) return Cnt(0.0);
  if (is_const(a.id, 1.0)) return b;
  if (is_const(b.id, 1.0)) return a;
  if (is_const(a.id, -1.0)) return Cnt(-b.v, vn('n', b.id, 0, nullptr));
  if (is_const(b.id, -1.0)) return Cnt(-a.v, vn('n', a.id, 0, nullptr));
  return Cnt(a.v * b.v, vn('*', a.id, b.id, &g.mul));
}
inline Cnt operator/(Cnt a, Cnt b) {
  if (is_const(b.id, 1.0)) return a;
  return Cnt(a.v / b.v, vn('/', a.id, b.id, &g.div));
}
inline Cnt operator-(Cnt a) { return Cnt(-a.v, vn('n', a.id, 0, nullptr)); }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
inline bool operator<(Cnt a, Cnt b) { return a.v < b.v; }
inline bool operator!=(Cnt a, Cnt b) { return a.v != b.v; }
inline Cnt sqrt(Cnt a) { return Cnt(std::sqrt(a.v), vn('s', a.id, 0, &g.sqrt)); }
inline Cnt exp(Cnt a) { return Cnt(std::exp(a.v), vn('e', a.id, 0, &g.exp)); }
inline Cnt erfc(Cnt a) { return Cnt(std::erfc(a.v), vn('c', a.id, 0, &g.erfc)); }
}  // namespace opc

#include "gks_point.cuh"

using opc::Cnt;
using namespace dghgks;

static int n_modes_(int k) { return (k + 1) * (k + 2) * (k + 3) / 6; }
static int n_tmodes_(int k) { return (k + 1) * (k + 2) / 2; }

// number of modes of P_k with a non-zero derivative along one axis
static int n_modes_dx(int k) {
  int c = 0;
  for (int a = 0; a <= k; ++a)
    for (int b = 0; a + b <= k; ++b)
      for (int d = 0; a + b + d <= k; ++d)
        if (a > 0) ++c;
  return c;
}

// A run-time input: a value with an id of its own, so that neither equal
// values nor zeros or ones among the inputs fold operations away.
static Cnt input(double x) { return Cnt(x, opc::next_id++); }

static void state(Cnt q[5], Cnt dq[3][5], double s) {
  const double rho = 1.1 + 0.1 * s, U = 0.3, V = -0.2, W = 0.1 + 0.1 * s, p = 71.4;
  q[0] = input(rho);
  q[1] = input(rho * U);
  q[2] = input(rho * V);
  q[3] = input(rho * W);
  q[4] = input(p / 0.4 + 0.5 * rho * (U * U + V * V + W * W));
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 5; ++k) dq[i][k] = input(0.01 * (1 + i + k) * (k == 4 ? 100.0 : 1.0));
}

static void emit(int order, int nq, double pr) {
  GasPar<Cnt> gp;
  gp.K = input(2.0);
  gp.gm1 = input(0.4);
  gp.mu = input(1.0 / 1600);
  gp.tau_add = input(0.0);
  gp.pr_fix = pr != 1.0 ? input(1.0 / pr - 1.0) : Cnt(0.0);  // the Pr = 1 kernels skip the heat terms
  gp.dt = input(3.3e-4);
  gp.inv_dt = input(1.0 / 3.3e-4);
  Cnt qL[5], dqL[3][5], qR[5], dqR[3][5], F[5], Ft[5], Fc[3][5], Ftc[3][5];
  state(qL, dqL, 0.0);
  state(qR, dqR, 1.0);
  opc::reset();
  iface_flux(qL, dqL, qR, dqR, gp, F, Ft);
  const opc::Tally face = opc::g;
  std::vector<int> outs;
  for (int k = 0; k < 5; ++k) outs.push_back(Ft[k].id);
  const opc::Tally face_ft = opc::live(outs);  // the S2O4 stage-2 pass needs F_t only
  opc::reset();
  interior_flux(qL, dqL, gp, Fc, Ftc);
  const opc::Tally cell = opc::g;
  outs.clear();
  for (int d = 0; d < 3; ++d)
    for (int k = 0; k < 5; ++k) outs.push_back(Ftc[d][k].id);
  const opc::Tally cell_ft = opc::live(outs);

  const int NM = n_modes_(order), NT = n_tmodes_(order), NMx = n_modes_dx(order), NN = n_tmodes_(order - 1);
  const int np = nq * nq;
  // Traces.  Basis factors P_0 = 1 and P'_1 = 1 are constants (folded);
  // a product of f non-constant factors takes f - 1 multiplies, a term
  // c * basis one FMA (2 flops), and the 3 x 5 gradients are scaled by 2/h.
  auto muls = [](int f) { return f > 1 ? f - 1 : 0; };
  // Face: per side and variable the value polynomial (NT tangential modes)
  // and the normal-derivative polynomial (NN) are formed once per face from
  // the cell's modes (a signed sum along the normal; factors n(n+1)/2 > 1
  // multiply) and evaluated at each point with the tangential basis and its
  // two derivatives (terms with P'_0 = 0 absent).
  long face_basis = 0, face_terms = 0;
  for (int a = 0; a <= order; ++a)
    for (int b = 0; a + b <= order; ++b) {
      face_basis += muls((a > 0) + (b > 0));
      face_terms += 1 + (a > 0) + (b > 0) + (a + b <= order - 1);
      if (a > 0) face_basis += muls((a > 1) + (b > 0));
      if (b > 0) face_basis += muls((a > 0) + (b > 1));
    }
  long collapse = 0;  // per side and variable, per face
  for (int m = 0, d = 0; d <= order; ++d)
    for (int a = 0; a <= order - d; ++a)
      for (int b = 0; a + b <= order - d; ++b, ++m) {
        (void)m;
        if (d > 0) collapse += 1;          // into the value polynomial (its first term is a move)
        if (d > 0 && d != 1) collapse += 1;  // n(n+1)/2 multiply
        if (d > 1) collapse += 1;            // into the normal polynomial
      }
  const long trace_face_side = 5 * face_terms * 2 + 15 + (5 * collapse + np - 1) / np;
  // Cell: per point and mode the value product and, per axis with a non-zero
  // exponent, the gradient product; one FMA per term.
  long cell_basis = 0, cell_terms = 0;
  for (int d = 0; d <= order; ++d)
    for (int a = 0; a + d <= order; ++a)
      for (int b = 0; a + b + d <= order; ++b) {
        const int e[3] = {d, a, b};
        cell_basis += muls((e[0] > 0) + (e[1] > 0) + (e[2] > 0));
        cell_terms += 1;
        for (int x = 0; x < 3; ++x)
          if (e[x] > 0) {
            cell_terms += 1;
            cell_basis += muls((e[x] > 1) + (e[(x + 1) % 3] > 0) + (e[(x + 2) % 3] > 0));
          }
      }
  const long trace_cell = cell_basis + 5 * cell_terms * 2 + 15;
  // face projection per point: 10 components x NT tangential modes FMA,
  // plus 10 weight multiplies
  const long proj_face = 10 * NT * 2 + 10;
  // cell projection per point: per direction only the NMx modes with a
  // non-zero derivative, 5 variables x (F, F_t) FMAs; plus 30 weight multiplies
  const long proj_cell = 3 * NMx * 5 * 2 * 2 + 30;
  const long face_total = face.flops() + face_basis + 2 * trace_face_side + proj_face;
  const long cell_total = cell.flops() + trace_cell + proj_cell;
  // F_t-only variants (stage 2 of S2O4): half of each projection
  const long face_total_ft = face_ft.flops() + face_basis + 2 * trace_face_side + 5 * NT * 2 + 5;
  const long cell_total_ft = cell_ft.flops() + trace_cell + 3 * NMx * 5 * 2 + 15;
  printf(
      "{\"order\": %d, \"n_q\": %d, \"pr_fix\": %s, "
      "\"face_point\": {\"flux_flops\": %ld, \"div\": %ld, \"sqrt\": %ld, \"exp\": %ld, \"erfc\": %ld, "
      "\"trace_flops\": %ld, \"proj_flops\": %ld, \"total_flops\": %ld, \"total_flops_ft\": %ld}, "
      "\"cell_point\": {\"flux_flops\": %ld, \"div\": %ld, \"sqrt\": %ld, \"exp\": %ld, \"erfc\": %ld, "
      "\"trace_flops\": %ld, \"proj_flops\": %ld, \"total_flops\": %ld, \"total_flops_ft\": %ld}}\n",
      order, nq, pr != 1.0 ? "true" : "false", face.flops(), face.div, face.sqrt, face.exp, face.erfc,
      face_basis + 2 * trace_face_side, proj_face, face_total, face_total_ft, cell.flops(), cell.div, cell.sqrt, cell.exp,
      cell.erfc, trace_cell, proj_cell, cell_total, cell_total_ft);
}

int main() {
  const int cfg[][2] = {{1, 2}, {2, 2}, {2, 3}, {3, 3}, {3, 4}};
  for (auto& c : cfg)
    for (double pr : {1.0, 0.72}) emit(c[0], c[1], pr);
  return 0;
}
