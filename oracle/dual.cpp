// Forward-mode derivative of the oracle's arithmetic (TEST INFRASTRUCTURE ONLY: the oracle's
// own derivative, against which the GPU adjoint is checked; the GPU library never uses it).
//
// orc2d.c is compiled here unchanged, with every `double` replaced by `dual`: a value and its
// derivative along one direction, propagated by the rules of differentiation (sum, product,
// quotient, square root; |x| and max(x, y) on the branch the values select). At the kink of |x|
// (x = 0) and of max(x, y) (x = y) the derivative is the mean of the two one-sided slopes (0
// for |x|, the mean of both derivatives for max): the value a central difference gives, and
// the one that keeps the characteristic splitting K^+ - K^- = A_k of eq. (int) consistent when
// a wave speed is exactly zero (a flow along the other direction). The values are the plain
// oracle's, operation for operation; elsewhere the derivatives are exact up to rounding. Arrays are pairs
// (value, derivative) per element; scalars are passed as such pairs by value.
#include <cmath>
#include <cstdlib>
#include <cstring>

struct dual {
  double v, d;
  dual() = default;
  dual(double x) : v(x), d(0.0) {}
  dual(double x, double dx) : v(x), d(dx) {}
  explicit operator int() const { return static_cast<int>(v); }
  explicit operator long() const { return static_cast<long>(v); }
};

inline dual operator+(dual a, dual b) { return dual(a.v + b.v, a.d + b.d); }
inline dual operator-(dual a, dual b) { return dual(a.v - b.v, a.d - b.d); }
inline dual operator*(dual a, dual b) { return dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline dual operator/(dual a, dual b) { return dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline dual operator-(dual a) { return dual(-a.v, -a.d); }
inline dual &operator+=(dual &a, dual b) { a = a + b; return a; }
inline dual &operator-=(dual &a, dual b) { a = a - b; return a; }
inline dual &operator*=(dual &a, dual b) { a = a * b; return a; }
inline dual &operator/=(dual &a, dual b) { a = a / b; return a; }
inline bool operator<(dual a, dual b) { return a.v < b.v; }
inline bool operator>(dual a, dual b) { return a.v > b.v; }
inline bool operator<=(dual a, dual b) { return a.v <= b.v; }
inline bool operator>=(dual a, dual b) { return a.v >= b.v; }
inline bool operator==(dual a, dual b) { return a.v == b.v; }
inline bool operator!=(dual a, dual b) { return a.v != b.v; }
inline dual sqrt(dual a) {
  const double r = std::sqrt(a.v);
  return dual(r, a.d / (2.0 * r));
}
inline dual fabs(dual a) { return a.v < 0.0 ? -a : (a.v > 0.0 ? a : dual(a.v, 0.0)); }
inline dual floor(dual a) { return dual(std::floor(a.v), 0.0); }
inline dual fmax(dual a, dual b) { return a.v > b.v ? a : (a.v < b.v ? b : dual(a.v, 0.5 * (a.d + b.d))); }

static_assert(sizeof(dual) == 2 * sizeof(double), "layout: (value, derivative) pairs");

#define double dual
extern "C" {
#include "orc2d.c"
}
#undef double
