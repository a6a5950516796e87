// Floating-point operation count of the oracle's per-point arithmetic (TEST INFRASTRUCTURE ONLY:
// the algorithmic FLOP count of a right-hand-side evaluation that the benchmark divides by the
// kernels' time for the FP64 roofline; the GPU library never uses it).
//
// orc2d.c is compiled here unchanged, with every `double` replaced by `fcount`, a value type
// that holds one double and adds one to a counter for each +, -, * and / and each square root it
// performs (comparisons, negation, fabs and floor count nothing). The oracle computes every
// intermediate once per point (full-array passes, no halos recomputed), so the count is the
// method's arithmetic as written, not that of any kernel design. fcount has the size, alignment
// and argument-passing class of double (a single double member), so the counting library takes
// the same arrays and scalars as the plain one through the same C signatures.
#include <cmath>
#include <cstdlib>
#include <cstring>

static unsigned long long g_flops = 0;

struct fcount {
  double v;
  fcount() = default;
  fcount(double x) : v(x) {}
  explicit operator int() const { return static_cast<int>(v); }
  explicit operator long() const { return static_cast<long>(v); }
};

inline fcount operator+(fcount a, fcount b) { ++g_flops; return fcount(a.v + b.v); }
inline fcount operator-(fcount a, fcount b) { ++g_flops; return fcount(a.v - b.v); }
inline fcount operator*(fcount a, fcount b) { ++g_flops; return fcount(a.v * b.v); }
inline fcount operator/(fcount a, fcount b) { ++g_flops; return fcount(a.v / b.v); }
inline fcount operator-(fcount a) { return fcount(-a.v); }
inline fcount &operator+=(fcount &a, fcount b) { a = a + b; return a; }
inline fcount &operator-=(fcount &a, fcount b) { a = a - b; return a; }
inline fcount &operator*=(fcount &a, fcount b) { a = a * b; return a; }
inline fcount &operator/=(fcount &a, fcount b) { a = a / b; return a; }
inline bool operator<(fcount a, fcount b) { return a.v < b.v; }
inline bool operator>(fcount a, fcount b) { return a.v > b.v; }
inline bool operator<=(fcount a, fcount b) { return a.v <= b.v; }
inline bool operator>=(fcount a, fcount b) { return a.v >= b.v; }
inline bool operator==(fcount a, fcount b) { return a.v == b.v; }
inline bool operator!=(fcount a, fcount b) { return a.v != b.v; }
inline fcount sqrt(fcount a) { ++g_flops; return fcount(std::sqrt(a.v)); }
inline fcount fabs(fcount a) { return fcount(std::fabs(a.v)); }
inline fcount floor(fcount a) { return fcount(std::floor(a.v)); }
inline fcount fmax(fcount a, fcount b) { return fcount(std::fmax(a.v, b.v)); }

static_assert(sizeof(fcount) == sizeof(double) && alignof(fcount) == alignof(double), "layout");

#define double fcount
extern "C" {
#include "orc2d.c"

unsigned long long orc_flops_read(int reset) {
  unsigned long long n = g_flops;
  if (reset) g_flops = 0;
  return n;
}
}
#undef double
