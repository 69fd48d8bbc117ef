/*
 * Scalar types of the oracle's two C++ builds (TEST INFRASTRUCTURE, like the
 * oracle itself).  aw_oracle.c is compiled once as plain C on double; the
 * translation units aw_oracle_tlm.cpp and aw_oracle_count.cpp compile the
 * same source with every `double` replaced by one of the types below, so the
 * arithmetic is the oracle's own, operation for operation:
 *
 *   dual     forward mode: (value, tangent) pairs; each operation applies the
 *            chain rule to the tangent.  Values are computed exactly as in the
 *            double build (same operations, no contraction), so comparisons,
 *            branches, floors and the integer schedule follow the plain run,
 *            and the tangent of an output is the directional derivative
 *            J'(x) v of the discrete map for the seeded input tangent v.
 *   opcount  the value plus a count of its floating-point operations: one per
 *            add, subtract, multiply, divide or square root (the oracle has
 *            no fused multiply-add), floor(log2 n) + popcount(n) - 1 for an
 *            integer power n (repeated squaring), none for comparisons,
 *            negation, absolute values, floor or min/max.  Counts go to the
 *            phase set by OC_PHASE.
 */
#ifndef OC_SCALAR_HPP
#define OC_SCALAR_HPP
#include <math.h>
#include <stdint.h>

struct dual {
  double v, d;
  dual() : v(0.0), d(0.0) {}
  dual(double x) : v(x), d(0.0) {}
  dual(double x, double dx) : v(x), d(dx) {}
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  explicit operator long long() const { return (long long)v; }
  dual& operator+=(const dual& b) { d += b.d; v += b.v; return *this; }
  dual& operator-=(const dual& b) { d -= b.d; v -= b.v; return *this; }
  dual& operator*=(const dual& b) { d = d * b.v + v * b.d; v *= b.v; return *this; }
  dual& operator/=(const dual& b) { const double q = v / b.v; d = (d - q * b.d) / b.v; v = q; return *this; }
};
inline dual operator+(const dual& a, const dual& b) { return dual(a.v + b.v, a.d + b.d); }
inline dual operator-(const dual& a, const dual& b) { return dual(a.v - b.v, a.d - b.d); }
inline dual operator*(const dual& a, const dual& b) { return dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline dual operator/(const dual& a, const dual& b) {
  const double q = a.v / b.v;
  return dual(q, (a.d - q * b.d) / b.v);
}
inline dual operator-(const dual& a) { return dual(-a.v, -a.d); }
inline bool operator<(const dual& a, const dual& b) { return a.v < b.v; }
inline bool operator>(const dual& a, const dual& b) { return a.v > b.v; }
inline bool operator<=(const dual& a, const dual& b) { return a.v <= b.v; }
inline bool operator>=(const dual& a, const dual& b) { return a.v >= b.v; }
inline bool operator==(const dual& a, const dual& b) { return a.v == b.v; }
inline bool operator!=(const dual& a, const dual& b) { return a.v != b.v; }
inline dual sqrt(const dual& a) {
  // a zero tangent stays zero, also at sqrt(0) (a vanishing norm)
  const double s = sqrt(a.v);
  return dual(s, a.d == 0.0 ? 0.0 : a.d / (2.0 * s));
}
inline dual fabs(const dual& a) { return a.v < 0.0 ? -a : a; }
inline dual floor(const dual& a) { return dual(floor(a.v), 0.0); }
inline dual fmax(const dual& a, const dual& b) { return a.v >= b.v ? a : b; }
inline dual cos(const dual& a) { return dual(cos(a.v), -sin(a.v) * a.d); }
inline dual ldexp(const dual& a, int e) { return dual(ldexp(a.v, e), ldexp(a.d, e)); }
inline dual pow(const dual& a, const dual& b) {
  // the oracle raises to constant exponents only (b.d == 0)
  const double p = pow(a.v, b.v);
  return dual(p, b.v * pow(a.v, b.v - 1.0) * a.d);
}

/* operation counts by phase */
enum { OC_PH_OTHER = 0, OC_PH_NODES, OC_PH_FLUX, OC_PH_UPDATE, OC_PH_RECON, OC_PH_DT, OC_PH_PRED, OC_PH_N };
extern int64_t oc_flops[OC_PH_N];
extern int oc_phase;

struct opcount {
  double v;
  static void tick(int64_t n = 1) { oc_flops[oc_phase] += n; }
  opcount() : v(0.0) {}
  opcount(double x) : v(x) {}
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  explicit operator long long() const { return (long long)v; }
  opcount& operator+=(const opcount& b) { tick(); v += b.v; return *this; }
  opcount& operator-=(const opcount& b) { tick(); v -= b.v; return *this; }
  opcount& operator*=(const opcount& b) { tick(); v *= b.v; return *this; }
  opcount& operator/=(const opcount& b) { tick(); v /= b.v; return *this; }
};
inline opcount operator+(const opcount& a, const opcount& b) { opcount::tick(); return opcount(a.v + b.v); }
inline opcount operator-(const opcount& a, const opcount& b) { opcount::tick(); return opcount(a.v - b.v); }
inline opcount operator*(const opcount& a, const opcount& b) { opcount::tick(); return opcount(a.v * b.v); }
inline opcount operator/(const opcount& a, const opcount& b) { opcount::tick(); return opcount(a.v / b.v); }
inline opcount operator-(const opcount& a) { return opcount(-a.v); }
inline bool operator<(const opcount& a, const opcount& b) { return a.v < b.v; }
inline bool operator>(const opcount& a, const opcount& b) { return a.v > b.v; }
inline bool operator<=(const opcount& a, const opcount& b) { return a.v <= b.v; }
inline bool operator>=(const opcount& a, const opcount& b) { return a.v >= b.v; }
inline bool operator==(const opcount& a, const opcount& b) { return a.v == b.v; }
inline bool operator!=(const opcount& a, const opcount& b) { return a.v != b.v; }
inline opcount sqrt(const opcount& a) { opcount::tick(); return opcount(sqrt(a.v)); }
inline opcount fabs(const opcount& a) { return opcount(fabs(a.v)); }
inline opcount floor(const opcount& a) { return opcount(floor(a.v)); }
inline opcount fmax(const opcount& a, const opcount& b) { return opcount(fmax(a.v, b.v)); }
inline opcount cos(const opcount& a) { opcount::tick(); return opcount(cos(a.v)); }
inline opcount ldexp(const opcount& a, int e) { return opcount(ldexp(a.v, e)); }
inline opcount pow(const opcount& a, const opcount& b) {
  const double e = b.v;
  if (e == floor(e) && e >= 1.0 && e < 64.0) {
    int n = (int)e, bits = 0, pc = 0;
    for (int k = n; k; k >>= 1) { ++bits; pc += k & 1; }
    opcount::tick(bits - 1 + pc - 1);
  } else {
    opcount::tick();
  }
  return opcount(pow(a.v, e));
}
#endif
