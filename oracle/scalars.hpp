// scalars.hpp — the two non-double scalar types the oracle is instantiated
// with.
//
// TEST INFRASTRUCTURE ONLY (see aerial_oracle.hpp).
//
//   Cnt  : a double that counts every floating-point operation applied to it.
//          Running one vehicle-step of the oracle in Cnt gives the
//          algorithmic operation count per vehicle-step used for the
//          roofline (adds/subs, muls, divs, square roots, transcendentals
//          and comparisons, each tallied separately; a sign flip is free).
//   Dual : a forward-mode dual number v + d*eps with eps^2 = 0. Running the
//          oracle's loss in Dual gives the exact directional derivative
//          (a Jacobian-vector product) of the FP64 loss, which checks the
//          hand-written adjoint independently of finite differences.
//   CntRev : a Cnt that also knows whether its value depends on the inputs
//          being differentiated ("active") and tallies, for every operation
//          with an active operand, the operations of that operation's
//          reverse-mode (adjoint) rule. Each rule accumulates into the
//          adjoint of every active operand, one addition per accumulation:
//            z = a +- b : a_bar += z_bar, b_bar +-= z_bar  (1 add per active operand)
//            z = a * b  : a_bar += z_bar b, b_bar += z_bar a  (1 mul + 1 add per active operand)
//            z = a / b  : t = z_bar / b (1 div); a_bar += t (1 add);
//                         b_bar -= t z (1 mul + 1 add)
//            z = sqrt a : a_bar += z_bar / (2 z)  (1 mul + 1 div + 1 add)
//            z = sin a, cos a : a_bar += z_bar (+-cos, sin) a  (1 trans + 1 mul + 1 add)
//            z = atan2(y, x) : r2 = x x + y y (2 mul + 1 add), t = z_bar / r2 (1 div),
//                         y_bar += t x, x_bar -= t y (1 mul + 1 add per active operand)
//          Sign flips and comparisons have no adjoint work. This is the
//          operation-by-operation reverse mode of automatic differentiation
//          (Griewank and Walther, "Evaluating Derivatives", 2nd ed., Ch. 3),
//          so running one step of the oracle in CntRev gives the algorithmic
//          operation count of one step of the rollout's adjoint.
#pragma once

#include <cmath>

namespace orc {

struct OpCounts { long long add, mul, div, sqrt, trans, cmp; };
inline OpCounts& op_counts() {
  static thread_local OpCounts c{0, 0, 0, 0, 0, 0};
  return c;
}

struct Cnt {
  double v;
  Cnt() : v(0.0) {}
  Cnt(double x) : v(x) {}  // NOLINT: implicit, so literals mix with Cnt
};
inline Cnt operator+(Cnt a, Cnt b) { op_counts().add++; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { op_counts().add++; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { op_counts().mul++; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { op_counts().div++; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline bool operator<(Cnt a, Cnt b) { op_counts().cmp++; return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { op_counts().cmp++; return a.v > b.v; }
inline bool operator==(Cnt a, Cnt b) { op_counts().cmp++; return a.v == b.v; }
inline Cnt sqrt(Cnt a) { op_counts().sqrt++; return Cnt(std::sqrt(a.v)); }
inline Cnt sin(Cnt a) { op_counts().trans++; return Cnt(std::sin(a.v)); }
inline Cnt cos(Cnt a) { op_counts().trans++; return Cnt(std::cos(a.v)); }
inline Cnt atan2(Cnt y, Cnt x) { op_counts().trans++; return Cnt(std::atan2(y.v, x.v)); }
inline double value_of(Cnt a) { return a.v; }

struct RevCounts { long long add, mul, div, sqrt, trans; };
inline RevCounts& rev_counts() {
  static thread_local RevCounts c{0, 0, 0, 0, 0};
  return c;
}

struct CntRev {
  double v;
  bool act;  // depends on a differentiated input
  CntRev() : v(0.0), act(false) {}
  CntRev(double x) : v(x), act(false) {}  // NOLINT: constants are inactive
  CntRev(double x, bool a) : v(x), act(a) {}
};
inline CntRev operator+(CntRev a, CntRev b) {
  op_counts().add++;
  rev_counts().add += (long long)a.act + (long long)b.act;
  return CntRev(a.v + b.v, a.act || b.act);
}
inline CntRev operator-(CntRev a, CntRev b) {
  op_counts().add++;
  rev_counts().add += (long long)a.act + (long long)b.act;
  return CntRev(a.v - b.v, a.act || b.act);
}
inline CntRev operator*(CntRev a, CntRev b) {
  op_counts().mul++;
  const long long n = (long long)a.act + (long long)b.act;
  rev_counts().mul += n;
  rev_counts().add += n;
  return CntRev(a.v * b.v, a.act || b.act);
}
inline CntRev operator/(CntRev a, CntRev b) {
  op_counts().div++;
  if (a.act || b.act) rev_counts().div++;
  if (a.act) rev_counts().add++;
  if (b.act) { rev_counts().mul++; rev_counts().add++; }
  return CntRev(a.v / b.v, a.act || b.act);
}
inline CntRev operator-(CntRev a) { return CntRev(-a.v, a.act); }
inline bool operator<(CntRev a, CntRev b) { op_counts().cmp++; return a.v < b.v; }
inline bool operator>(CntRev a, CntRev b) { op_counts().cmp++; return a.v > b.v; }
inline bool operator==(CntRev a, CntRev b) { op_counts().cmp++; return a.v == b.v; }
inline CntRev sqrt(CntRev a) {
  op_counts().sqrt++;
  if (a.act) { rev_counts().mul++; rev_counts().div++; rev_counts().add++; }
  return CntRev(std::sqrt(a.v), a.act);
}
inline CntRev sin(CntRev a) {
  op_counts().trans++;
  if (a.act) { rev_counts().trans++; rev_counts().mul++; rev_counts().add++; }
  return CntRev(std::sin(a.v), a.act);
}
inline CntRev cos(CntRev a) {
  op_counts().trans++;
  if (a.act) { rev_counts().trans++; rev_counts().mul++; rev_counts().add++; }
  return CntRev(std::cos(a.v), a.act);
}
inline CntRev atan2(CntRev y, CntRev x) {
  op_counts().trans++;
  const long long n = (long long)y.act + (long long)x.act;
  if (n > 0) {
    rev_counts().mul += 2 + n;
    rev_counts().add += 1 + n;
    rev_counts().div++;
  }
  return CntRev(std::atan2(y.v, x.v), y.act || x.act);
}
inline double value_of(CntRev a) { return a.v; }

struct Dual {
  double v, d;
  Dual() : v(0.0), d(0.0) {}
  Dual(double x) : v(x), d(0.0) {}  // NOLINT: constants carry no tangent
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
inline Dual sqrt(Dual a) { double r = std::sqrt(a.v); return Dual(r, a.d / (2.0 * r)); }
inline Dual sin(Dual a) { return Dual(std::sin(a.v), std::cos(a.v) * a.d); }
inline Dual cos(Dual a) { return Dual(std::cos(a.v), -std::sin(a.v) * a.d); }
inline Dual atan2(Dual y, Dual x) {
  double r2 = x.v * x.v + y.v * y.v;
  return Dual(std::atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / r2);
}
inline double value_of(Dual a) { return a.v; }
inline double value_of(double a) { return a; }

}  // namespace orc
