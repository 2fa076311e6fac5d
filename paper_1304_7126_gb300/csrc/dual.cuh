// First-order dual numbers v + d eps (eps^2 = 0) for forward-mode
// differentiation of the per-cell thermochemistry.
//
// The thermochemistry code is templated on its scalar type; instantiated
// with Dual it carries, next to every value, the derivative of that value
// along one seeded input direction.  The value parts go through exactly the
// operations of the double instantiation (same order, same operands), so
// the sub-cycle decisions of the 10% rule, taken on values, are those of
// the FP64 forward kernels.  Comparisons, min/max and |.| act on values;
// min/max/|.| pass the derivative of the branch they take.
#pragma once

#include <cuda_runtime.h>

namespace rtgb {

// the double overloads stay visible next to the Dual ones below
using ::exp;
using ::fabs;
using ::fma;
using ::fmax;
using ::fmin;
using ::log;
using ::log1p;
using ::sqrt;

struct Dual {
    double v, d;
    Dual() = default;
    __host__ __device__ constexpr Dual(double x) : v(x), d(0.0) {}
    __host__ __device__ constexpr Dual(double x, double dx) : v(x), d(dx) {}
};

__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(const Dual &x) { return x.v; }

__device__ __forceinline__ Dual operator-(const Dual &a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator+(const Dual &a, const Dual &b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator+(const Dual &a, double b) { return Dual(a.v + b, a.d); }
__device__ __forceinline__ Dual operator+(double a, const Dual &b) { return Dual(a + b.v, b.d); }
__device__ __forceinline__ Dual operator-(const Dual &a, const Dual &b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(const Dual &a, double b) { return Dual(a.v - b, a.d); }
__device__ __forceinline__ Dual operator-(double a, const Dual &b) { return Dual(a - b.v, -b.d); }
__device__ __forceinline__ Dual operator*(const Dual &a, const Dual &b)
{
    return Dual(a.v * b.v, a.d * b.v + a.v * b.d);
}
__device__ __forceinline__ Dual operator*(const Dual &a, double b) { return Dual(a.v * b, a.d * b); }
__device__ __forceinline__ Dual operator*(double a, const Dual &b) { return Dual(a * b.v, a * b.d); }
__device__ __forceinline__ Dual operator/(const Dual &a, const Dual &b)
{
    const double q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ Dual operator/(const Dual &a, double b) { return Dual(a.v / b, a.d / b); }
__device__ __forceinline__ Dual operator/(double a, const Dual &b)
{
    const double q = a / b.v;
    return Dual(q, -q * b.d / b.v);
}
// products and sums rounded as written (never fused into an FMA): the
// value of a dual is then bit for bit the double computed the same way
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ Dual rmul(const Dual &a, const Dual &b)
{
    return Dual(__dmul_rn(a.v, b.v), a.v * b.d + a.d * b.v);
}
__device__ __forceinline__ Dual rmul(const Dual &a, double b) { return Dual(__dmul_rn(a.v, b), a.d * b); }
__device__ __forceinline__ Dual radd(const Dual &a, const Dual &b) { return Dual(__dadd_rn(a.v, b.v), a.d + b.d); }
// a b + c with one rounding, as written
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ Dual rfma(double a, const Dual &b, const Dual &c)
{
    return Dual(__fma_rn(a, b.v, c.v), a * b.d + c.d);
}
__device__ __forceinline__ Dual rfma(const Dual &a, const Dual &b, const Dual &c)
{
    return Dual(__fma_rn(a.v, b.v, c.v), a.d * b.v + a.v * b.d + c.d);
}

__device__ __forceinline__ Dual &operator+=(Dual &a, const Dual &b) { a = a + b; return a; }
__device__ __forceinline__ Dual &operator-=(Dual &a, const Dual &b) { a = a - b; return a; }
__device__ __forceinline__ Dual &operator*=(Dual &a, const Dual &b) { a = a * b; return a; }

#define RTGB_DUAL_CMP(op)                                                                              \
    __device__ __forceinline__ bool operator op(const Dual &a, const Dual &b) { return a.v op b.v; } \
    __device__ __forceinline__ bool operator op(const Dual &a, double b) { return a.v op b; }         \
    __device__ __forceinline__ bool operator op(double a, const Dual &b) { return a op b.v; }
RTGB_DUAL_CMP(<)
RTGB_DUAL_CMP(>)
RTGB_DUAL_CMP(<=)
RTGB_DUAL_CMP(>=)
RTGB_DUAL_CMP(==)
RTGB_DUAL_CMP(!=)
#undef RTGB_DUAL_CMP

__device__ __forceinline__ Dual fma(const Dual &a, const Dual &b, const Dual &c)
{
    return Dual(::fma(a.v, b.v, c.v), a.d * b.v + a.v * b.d + c.d);
}
__device__ __forceinline__ Dual fabs(const Dual &a) { return a.v < 0.0 ? -a : a; }
__device__ __forceinline__ Dual fmin(const Dual &a, const Dual &b) { return (b.v < a.v) ? b : a; }
__device__ __forceinline__ Dual fmin(const Dual &a, double b) { return (b < a.v) ? Dual(b) : a; }
__device__ __forceinline__ Dual fmax(const Dual &a, const Dual &b) { return (b.v > a.v) ? b : a; }
__device__ __forceinline__ Dual fmax(const Dual &a, double b) { return (b > a.v) ? Dual(b) : a; }
__device__ __forceinline__ Dual fmax(double a, const Dual &b) { return (b.v > a) ? b : Dual(a); }
__device__ __forceinline__ Dual sqrt(const Dual &a)
{
    const double r = ::sqrt(a.v);
    return Dual(r, r > 0.0 ? 0.5 * a.d / r : 0.0);
}
__device__ __forceinline__ Dual exp(const Dual &a)
{
    const double e = ::exp(a.v);
    return Dual(e, e * a.d);
}
__device__ __forceinline__ Dual log(const Dual &a) { return Dual(::log(a.v), a.d / a.v); }
__device__ __forceinline__ Dual log1p(const Dual &a) { return Dual(::log1p(a.v), a.d / (1.0 + a.v)); }


}  // namespace rtgb
