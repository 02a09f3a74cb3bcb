/* Operation-counting stand-in for double, used only by the counting build of
 * the CPU oracle (compiled with -DORACLE_COUNT_FLOPS).  Every +, -, *, / and
 * sqrt on a `real` adds one to a per-kind counter; comparisons, min/max and
 * fabs are tallied separately because they are not floating-point arithmetic.
 * Test infrastructure only. */
#ifndef ORACLE_FLOPCOUNT_H
#define ORACLE_FLOPCOUNT_H
#include <cmath>

struct op_tally { long long add, mul, div, sqrt, cmp; };
extern op_tally g_tally;

struct counted {
  double v;
  counted() : v(0.0) {}
  counted(double x) : v(x) {}
  explicit operator double() const { return v; }
  counted operator-() const { return counted(-v); }
  counted& operator+=(counted o) { ++g_tally.add; v += o.v; return *this; }
  counted& operator-=(counted o) { ++g_tally.add; v -= o.v; return *this; }
};
inline counted operator+(counted a, counted b) { ++g_tally.add; return counted(a.v + b.v); }
inline counted operator-(counted a, counted b) { ++g_tally.add; return counted(a.v - b.v); }
inline counted operator*(counted a, counted b) { ++g_tally.mul; return counted(a.v * b.v); }
inline counted operator/(counted a, counted b) { ++g_tally.div; return counted(a.v / b.v); }
inline counted operator+(double a, counted b) { ++g_tally.add; return counted(a + b.v); }
inline counted operator-(double a, counted b) { ++g_tally.add; return counted(a - b.v); }
inline counted operator*(double a, counted b) { ++g_tally.mul; return counted(a * b.v); }
inline counted operator/(double a, counted b) { ++g_tally.div; return counted(a / b.v); }
inline counted operator+(counted a, double b) { ++g_tally.add; return counted(a.v + b); }
inline counted operator-(counted a, double b) { ++g_tally.add; return counted(a.v - b); }
inline counted operator*(counted a, double b) { ++g_tally.mul; return counted(a.v * b); }
inline counted operator/(counted a, double b) { ++g_tally.div; return counted(a.v / b); }
#define CMP_OP(op) \
  inline bool operator op(counted a, counted b) { ++g_tally.cmp; return a.v op b.v; } \
  inline bool operator op(counted a, double b) { ++g_tally.cmp; return a.v op b; } \
  inline bool operator op(double a, counted b) { ++g_tally.cmp; return a op b.v; }
CMP_OP(<) CMP_OP(>) CMP_OP(<=) CMP_OP(>=) CMP_OP(==) CMP_OP(!=)
#undef CMP_OP
inline counted sqrt(counted a) { ++g_tally.sqrt; return counted(std::sqrt(a.v)); }
inline counted fabs(counted a) { return counted(std::fabs(a.v)); }
inline counted copysign(counted a, counted b) { return counted(std::copysign(a.v, b.v)); }
inline bool isfinite(counted a) { return std::isfinite(a.v); }
#endif
