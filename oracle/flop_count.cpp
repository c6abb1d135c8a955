/*
 * flop_count.cpp -- the oracle (sse_oracle.c) compiled once more, unchanged,
 * with every `double` replaced by om_f64: an 8-byte wrapper whose arithmetic
 * operators perform the same IEEE double operation and add one to a counter.
 *
 * TEST INFRASTRUCTURE ONLY, like the oracle itself.  It measures the
 * algorithmic floating-point work of the method as the oracle writes it (one
 * count per +, -, *, / and sqrt on FP64 values; sign changes, comparisons,
 * fabs and conversions count nothing; a product followed by a sum counts two,
 * as an FMA does).  The library exports the oracle's entry points plus
 * om_flops_reset / om_flops_read; its results are bit-identical to the plain
 * build's (both compiled without FMA contraction, the same operations in the
 * same order), which tests/test_oracle_flops.py checks together with exact
 * counts of operators whose work is known in closed form.  Serial only.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>

static unsigned long long g_om_flops = 0;

struct om_f64 {
    double v;
    om_f64() = default;
    om_f64(double x) : v(x) {}
    // no implicit conversion back to double: every arithmetic use of a value
    // must go through the counting operators below
    explicit operator double() const { return v; }
    explicit operator bool() const { return v != 0.0; }
    om_f64 &operator+=(om_f64 b) { ++g_om_flops; v += b.v; return *this; }
    om_f64 &operator-=(om_f64 b) { ++g_om_flops; v -= b.v; return *this; }
    om_f64 &operator*=(om_f64 b) { ++g_om_flops; v *= b.v; return *this; }
    om_f64 &operator/=(om_f64 b) { ++g_om_flops; v /= b.v; return *this; }
};
static_assert(sizeof(om_f64) == sizeof(double) && alignof(om_f64) == alignof(double),
              "om_f64 has the layout of double (the arrays come from numpy)");
static_assert(std::is_trivially_copyable<om_f64>::value, "om_f64 copies like double");

template <class T>
using om_num = std::enable_if_t<std::is_arithmetic<T>::value, int>;

#define OM_ARITH(op)                                                                         \
    inline om_f64 operator op(om_f64 a, om_f64 b) { ++g_om_flops; return a.v op b.v; }      \
    template <class T, om_num<T> = 0> inline om_f64 operator op(om_f64 a, T b) {            \
        ++g_om_flops;                                                                        \
        return a.v op (double)b;                                                             \
    }                                                                                        \
    template <class T, om_num<T> = 0> inline om_f64 operator op(T a, om_f64 b) {            \
        ++g_om_flops;                                                                        \
        return (double)a op b.v;                                                             \
    }
OM_ARITH(+)
OM_ARITH(-)
OM_ARITH(*)
OM_ARITH(/)
#undef OM_ARITH

#define OM_CMP(op)                                                                           \
    inline bool operator op(om_f64 a, om_f64 b) { return a.v op b.v; }                       \
    template <class T, om_num<T> = 0> inline bool operator op(om_f64 a, T b) {              \
        return a.v op (double)b;                                                             \
    }                                                                                        \
    template <class T, om_num<T> = 0> inline bool operator op(T a, om_f64 b) {              \
        return (double)a op b.v;                                                             \
    }
OM_CMP(<)
OM_CMP(>)
OM_CMP(<=)
OM_CMP(>=)
OM_CMP(==)
OM_CMP(!=)
#undef OM_CMP

inline om_f64 operator-(om_f64 a) { return -a.v; }
inline om_f64 operator+(om_f64 a) { return a; }
inline om_f64 sqrt(om_f64 a) { ++g_om_flops; return ::sqrt(a.v); }
inline om_f64 fabs(om_f64 a) { return ::fabs(a.v); }

// the oracle's source, every double an om_f64 (its header keeps C linkage)
#define double om_f64
#include "sse_oracle.c"
#undef double

extern "C" void om_flops_reset(void) { g_om_flops = 0; }
extern "C" unsigned long long om_flops_read(void) { return g_om_flops; }
