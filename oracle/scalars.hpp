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
inline Cnt sqrt(Cnt a) { op_counts().sqrt++; return Cnt(std::sqrt(a.v)); }
inline Cnt sin(Cnt a) { op_counts().trans++; return Cnt(std::sin(a.v)); }
inline Cnt cos(Cnt a) { op_counts().trans++; return Cnt(std::cos(a.v)); }
inline Cnt atan2(Cnt y, Cnt x) { op_counts().trans++; return Cnt(std::atan2(y.v, x.v)); }
inline double value_of(Cnt a) { return a.v; }

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
