/* ora_real.h -- scalar type of the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY. The oracle is the plain FP64 reference that the
 * CUDA path is checked against; nothing in the product links it.
 *
 * By default `real` is `double`. Built with -DORA_COUNT_FLOPS, `real` becomes
 * a thin wrapper that counts the floating-point operations it performs, so the
 * oracle itself states the algorithmic FP64 cost of one zone-cycle
 * (add/sub/mul, divisions, square roots, transcendentals, compares).
 * An add/sub or mul with an operand that is exactly zero is not counted: the
 * oracle contracts full 4x4 metrics, and the zero entries of the Kerr-Schild
 * metric are not work the method needs to do.
 */
#ifndef ORA_REAL_H
#define ORA_REAL_H

#include <cmath>

#ifndef ORA_COUNT_FLOPS

typedef double real;
static inline double tod(double x) { return x; }
using std::isfinite;

#else

/* counters: 0 add/sub/mul, 1 div, 2 sqrt, 3 exp/log/pow, 4 compare/min/max */
extern "C" unsigned long long ora_flop_ctr[5];

struct real {
    double v;
    real() : v(0.0) {}
    real(double x) : v(x) {}
    real(int x) : v((double)x) {}
    real& operator+=(const real& o) { if (v != 0.0 && o.v != 0.0) ora_flop_ctr[0]++; v += o.v; return *this; }
    real& operator-=(const real& o) { if (v != 0.0 && o.v != 0.0) ora_flop_ctr[0]++; v -= o.v; return *this; }
    real& operator*=(const real& o) { if (v != 0.0 && o.v != 0.0) ora_flop_ctr[0]++; v *= o.v; return *this; }
    real& operator/=(const real& o) { ora_flop_ctr[1]++; v /= o.v; return *this; }
    real operator-() const { return real(-v); }
};
static inline double tod(const real& x) { return x.v; }
static inline void ora_cnt2(double a, double b) { if (a != 0.0 && b != 0.0) ora_flop_ctr[0]++; }
static inline real operator+(const real& a, const real& b) { ora_cnt2(a.v, b.v); return real(a.v + b.v); }
static inline real operator-(const real& a, const real& b) { ora_cnt2(a.v, b.v); return real(a.v - b.v); }
static inline real operator*(const real& a, const real& b) { ora_cnt2(a.v, b.v); return real(a.v * b.v); }
static inline real operator/(const real& a, const real& b) { ora_flop_ctr[1]++; return real(a.v / b.v); }
static inline real operator+(const real& a, double b) { ora_cnt2(a.v, b); return real(a.v + b); }
static inline real operator-(const real& a, double b) { ora_cnt2(a.v, b); return real(a.v - b); }
static inline real operator*(const real& a, double b) { ora_cnt2(a.v, b); return real(a.v * b); }
static inline real operator/(const real& a, double b) { ora_flop_ctr[1]++; return real(a.v / b); }
static inline real operator+(double a, const real& b) { ora_cnt2(a, b.v); return real(a + b.v); }
static inline real operator-(double a, const real& b) { ora_cnt2(a, b.v); return real(a - b.v); }
static inline real operator*(double a, const real& b) { ora_cnt2(a, b.v); return real(a * b.v); }
static inline real operator/(double a, const real& b) { ora_flop_ctr[1]++; return real(a / b.v); }
#define ORA_CMP(op)                                                                          \
    static inline bool operator op(const real& a, const real& b) { ora_flop_ctr[4]++; return a.v op b.v; } \
    static inline bool operator op(const real& a, double b) { ora_flop_ctr[4]++; return a.v op b; }        \
    static inline bool operator op(double a, const real& b) { ora_flop_ctr[4]++; return a op b.v; }
ORA_CMP(<) ORA_CMP(>) ORA_CMP(<=) ORA_CMP(>=) ORA_CMP(==) ORA_CMP(!=)
#undef ORA_CMP
static inline real sqrt(const real& a) { ora_flop_ctr[2]++; return real(std::sqrt(a.v)); }
static inline real fabs(const real& a) { return real(std::fabs(a.v)); }
static inline real exp(const real& a) { ora_flop_ctr[3]++; return real(std::exp(a.v)); }
static inline real log(const real& a) { ora_flop_ctr[3]++; return real(std::log(a.v)); }
static inline real pow(const real& a, const real& b) { ora_flop_ctr[3]++; return real(std::pow(a.v, b.v)); }
static inline real pow(const real& a, double b) { ora_flop_ctr[3]++; return real(std::pow(a.v, b)); }
static inline real acos(const real& a) { ora_flop_ctr[3]++; return real(std::acos(a.v)); }
static inline real cos(const real& a) { ora_flop_ctr[3]++; return real(std::cos(a.v)); }
static inline real cbrt(const real& a) { ora_flop_ctr[3]++; return real(std::cbrt(a.v)); }
static inline real fmax(const real& a, const real& b) { ora_flop_ctr[4]++; return real(std::fmax(a.v, b.v)); }
static inline real fmin(const real& a, const real& b) { ora_flop_ctr[4]++; return real(std::fmin(a.v, b.v)); }
static inline real fmax(const real& a, double b) { ora_flop_ctr[4]++; return real(std::fmax(a.v, b)); }
static inline real fmin(const real& a, double b) { ora_flop_ctr[4]++; return real(std::fmin(a.v, b)); }
static inline real fmax(double a, const real& b) { ora_flop_ctr[4]++; return real(std::fmax(a, b.v)); }
static inline real fmin(double a, const real& b) { ora_flop_ctr[4]++; return real(std::fmin(a, b.v)); }
static inline bool isfinite(const real& a) { return std::isfinite(a.v); }

#endif /* ORA_COUNT_FLOPS */

#endif /* ORA_REAL_H */
