// ORACLE -- test and measurement infrastructure only.  The counting scalar of
// the op-counting build (opcount.cpp): a double whose arithmetic operations
// increment hwo_ops (add/sub, mul, div, sqrt, pow).
#pragma once
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>

extern unsigned long long hwo_ops[5];  // add/sub, mul, div, sqrt, pow

struct hwo_real {
  double v;
  hwo_real() = default;
  constexpr hwo_real(double x) : v(x) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return (int)v; }
  hwo_real& operator+=(hwo_real b) { ++hwo_ops[0]; v += b.v; return *this; }
  hwo_real& operator-=(hwo_real b) { ++hwo_ops[0]; v -= b.v; return *this; }
  hwo_real& operator*=(hwo_real b) { ++hwo_ops[1]; v *= b.v; return *this; }
  hwo_real& operator/=(hwo_real b) { ++hwo_ops[2]; v /= b.v; return *this; }
};
static_assert(sizeof(hwo_real) == sizeof(double), "the layout of a double");

inline hwo_real operator+(hwo_real a, hwo_real b) { ++hwo_ops[0]; return a.v + b.v; }
inline hwo_real operator-(hwo_real a, hwo_real b) { ++hwo_ops[0]; return a.v - b.v; }
inline hwo_real operator*(hwo_real a, hwo_real b) { ++hwo_ops[1]; return a.v * b.v; }
inline hwo_real operator/(hwo_real a, hwo_real b) { ++hwo_ops[2]; return a.v / b.v; }
inline hwo_real operator-(hwo_real a) { return -a.v; }
inline hwo_real operator+(hwo_real a) { return a; }
inline bool operator<(hwo_real a, hwo_real b) { return a.v < b.v; }
inline bool operator>(hwo_real a, hwo_real b) { return a.v > b.v; }
inline bool operator<=(hwo_real a, hwo_real b) { return a.v <= b.v; }
inline bool operator>=(hwo_real a, hwo_real b) { return a.v >= b.v; }
inline bool operator==(hwo_real a, hwo_real b) { return a.v == b.v; }
inline bool operator!=(hwo_real a, hwo_real b) { return a.v != b.v; }
inline hwo_real sqrt(hwo_real a) { ++hwo_ops[3]; return std::sqrt(a.v); }
inline hwo_real fabs(hwo_real a) { return std::fabs(a.v); }
inline hwo_real pow(hwo_real a, hwo_real b) { ++hwo_ops[4]; return std::pow(a.v, b.v); }
inline hwo_real pow(hwo_real a, int b) { ++hwo_ops[4]; return std::pow(a.v, b); }

