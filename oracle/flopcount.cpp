// Test infrastructure (like the rest of oracle/): counts the floating-point
// operations of the oracle's RK4 step per interior cell and stage, i.e. the
// algorithmic flops of the method as the oracle writes it out (right-hand
// side with its centred, mixed, lopsided and KO stencils, the RK4 stage
// update, the algebraic enforcement).  The oracle's own C source is compiled
// with `double` replaced by a counting scalar: every +, -, * on it counts
// one operation, divisions, square roots and powers are tallied separately.
// The oracle has no fused multiply-adds (it is built with
// -ffp-contract=off), so nothing is counted twice.
//
// Build and run: see oracle/flopcount.py.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

namespace fc {
struct Tally {
  long long add = 0, mul = 0, div = 0, sqrt_ = 0, pow_ = 0;
};
static Tally T;
static bool on = false;

struct D {
  double v;
  D() = default;
  constexpr D(double x) : v(x) {}
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  explicit operator long long() const { return (long long)v; }
  explicit operator char() const { return (char)v; }
};
inline D operator+(D a, D b) { T.add += on; return D(a.v + b.v); }
inline D operator-(D a, D b) { T.add += on; return D(a.v - b.v); }
inline D operator*(D a, D b) { T.mul += on; return D(a.v * b.v); }
inline D operator/(D a, D b) { T.div += on; return D(a.v / b.v); }
inline D operator-(D a) { return D(-a.v); }
inline D operator+(D a) { return a; }
inline D &operator+=(D &a, D b) { a = a + b; return a; }
inline D &operator-=(D &a, D b) { a = a - b; return a; }
inline D &operator*=(D &a, D b) { a = a * b; return a; }
inline D &operator/=(D &a, D b) { a = a / b; return a; }
inline bool operator<(D a, D b) { return a.v < b.v; }
inline bool operator>(D a, D b) { return a.v > b.v; }
inline bool operator<=(D a, D b) { return a.v <= b.v; }
inline bool operator>=(D a, D b) { return a.v >= b.v; }
inline bool operator==(D a, D b) { return a.v == b.v; }
inline bool operator!=(D a, D b) { return a.v != b.v; }
inline D sqrt(D a) { T.sqrt_ += on; return D(::sqrt(a.v)); }
inline D pow(D a, D b) { T.pow_ += on; return D(::pow(a.v, b.v)); }
inline D fabs(D a) { return D(::fabs(a.v)); }
inline D floor(D a) { return D(::floor(a.v)); }
inline D ceil(D a) { return D(::ceil(a.v)); }
inline long long llround(D a) { return ::llround(a.v); }
inline D sin(D a) { return D(::sin(a.v)); }
inline D cos(D a) { return D(::cos(a.v)); }
inline D log(D a) { return D(::log(a.v)); }
}  // namespace fc

#define double fc::D
#include "z4c_oracle.c"
#undef double

// One block of n^3 interior cells, periodic (no Sommerfeld cells), order and
// ghosts as given, smooth generic data; one RK4 step counted.
int main(int argc, char **argv) {
  const int order = argc > 1 ? atoi(argv[1]) : 6;
  const int n = 8, g = order / 2 + 1;
  orc_mesh m;
  memset((void *)&m, 0, sizeof m);
  int32_t nn[3] = {n, n, n};
  fc::D lo[3] = {-0.5, -0.5, -0.5}, h[1] = {1.0 / n};
  m.nblocks = 1;
  m.ghosts = g;
  m.order = order;
  m.n = nn;
  m.lo = lo;
  m.h = h;
  for (int d = 0; d < 3; ++d) {
    m.dom_lo[d] = -0.5;
    m.dom_hi[d] = 0.5;
  }
  m.periodic = 1;
  m.lapse = 1;
  m.shift = 1;
  m.ko_sigma = 0.5;
  m.kappa1 = 0.02;
  m.kappa2 = 0.0;
  m.eta = 2.0;
  m.chi_floor = 1e-6;
  const long size = orc_state_size(&m);
  fc::D *u = (fc::D *)malloc(sizeof(fc::D) * size);
  const long e = n + 2 * g, S = e * e * e;
  // a generic smooth state (a perturbed flat metric; every term of the RHS is
  // exercised, none of it is special-cased by value)
  for (int f = 0; f < NF; ++f)
    for (long c = 0; c < S; ++c) {
      const double x = (double)(c % e) / e, y = (double)((c / e) % e) / e, z = (double)(c / (e * e)) / e;
      double v = 0.01 * ::sin(6.283 * x + f) * ::cos(6.283 * y - 0.3 * f) + 0.005 * ::sin(6.283 * z + 0.1 * f);
      if (f == F_CHI || f == F_ALPHA || f == F_GXX || f == F_GYY || f == F_GZZ) v += 1.0;
      u[(long)f * S + c] = v;
    }
  fc::on = true;
  const int rc = orc_rk4_step(&m, u, 0.01, 1);
  fc::on = false;
  const double cells_stages = 4.0 * n * n * n;
  printf("{\"order\": %d, \"rc\": %d, \"add\": %.1f, \"mul\": %.1f, \"div\": %.2f, \"sqrt\": %.3f, \"pow\": %.3f, "
         "\"flops_per_cell_stage\": %.1f}\n",
         order, rc, fc::T.add / cells_stages, fc::T.mul / cells_stages, fc::T.div / cells_stages,
         fc::T.sqrt_ / cells_stages, fc::T.pow_ / cells_stages, (fc::T.add + fc::T.mul) / cells_stages);
  free(u);
  return rc;
}
