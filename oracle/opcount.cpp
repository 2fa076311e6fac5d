// Op-counting build of the oracle (test and measurement infrastructure, like
// the oracle itself): rt_oracle.c compiled as C++ with every double replaced
// by OpDouble, a scalar with the layout of a double that counts the
// floating-point operations the oracle's statement of the method performs.
// It runs the oracle's own code, so the counts are the algorithmic work of
// the step as the paper's method states it (App. A, Sec. 3.2), independent
// of how the CUDA library arranges that work.
//
// Counted: additions and subtractions, multiplications, divisions, square
// roots (one flop each), and calls of exp, log and pow (reported apart).
// Comparisons, fabs, fmin, fmax, floor and negation are not counted.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

namespace opcount {
struct Counts {
    unsigned long long add, mul, div, sqrt, exp, log, pow;
};
Counts g;
}  // namespace opcount

struct OpDouble {
    double v;
    OpDouble() = default;
    OpDouble(double x) : v(x) {}
    explicit operator double() const { return v; }
    explicit operator int() const { return (int)v; }
    OpDouble &operator+=(OpDouble b) { ++opcount::g.add; v += b.v; return *this; }
    OpDouble &operator-=(OpDouble b) { ++opcount::g.add; v -= b.v; return *this; }
    OpDouble &operator*=(OpDouble b) { ++opcount::g.mul; v *= b.v; return *this; }
    OpDouble &operator/=(OpDouble b) { ++opcount::g.div; v /= b.v; return *this; }
    OpDouble operator-() const { return OpDouble(-v); }
};
static_assert(sizeof(OpDouble) == sizeof(double), "same layout as a double");

static inline OpDouble operator+(OpDouble a, OpDouble b) { ++opcount::g.add; return OpDouble(a.v + b.v); }
static inline OpDouble operator-(OpDouble a, OpDouble b) { ++opcount::g.add; return OpDouble(a.v - b.v); }
static inline OpDouble operator*(OpDouble a, OpDouble b) { ++opcount::g.mul; return OpDouble(a.v * b.v); }
static inline OpDouble operator/(OpDouble a, OpDouble b) { ++opcount::g.div; return OpDouble(a.v / b.v); }
static inline bool operator<(OpDouble a, OpDouble b) { return a.v < b.v; }
static inline bool operator>(OpDouble a, OpDouble b) { return a.v > b.v; }
static inline bool operator<=(OpDouble a, OpDouble b) { return a.v <= b.v; }
static inline bool operator>=(OpDouble a, OpDouble b) { return a.v >= b.v; }
static inline bool operator==(OpDouble a, OpDouble b) { return a.v == b.v; }
static inline bool operator!=(OpDouble a, OpDouble b) { return a.v != b.v; }
static inline OpDouble sqrt(OpDouble a) { ++opcount::g.sqrt; return OpDouble(::sqrt(a.v)); }
static inline OpDouble exp(OpDouble a) { ++opcount::g.exp; return OpDouble(::exp(a.v)); }
static inline OpDouble log(OpDouble a) { ++opcount::g.log; return OpDouble(::log(a.v)); }
static inline OpDouble pow(OpDouble a, OpDouble b) { ++opcount::g.pow; return OpDouble(::pow(a.v, b.v)); }
static inline OpDouble fabs(OpDouble a) { return OpDouble(::fabs(a.v)); }
static inline OpDouble fmax(OpDouble a, OpDouble b) { return OpDouble(::fmax(a.v, b.v)); }
static inline OpDouble fmin(OpDouble a, OpDouble b) { return OpDouble(::fmin(a.v, b.v)); }
static inline OpDouble floor(OpDouble a) { return OpDouble(::floor(a.v)); }
static inline OpDouble ldexp(OpDouble a, int e) { return OpDouble(::ldexp(a.v, e)); }

#define double OpDouble
extern "C" {
#include "rt_oracle.c"
}
#undef double

extern "C" void oracle_opcount_get(unsigned long long *out)
{
    const opcount::Counts &c = opcount::g;
    out[0] = c.add;
    out[1] = c.mul;
    out[2] = c.div;
    out[3] = c.sqrt;
    out[4] = c.exp;
    out[5] = c.log;
    out[6] = c.pow;
}

extern "C" void oracle_opcount_reset(void) { opcount::g = opcount::Counts{}; }
