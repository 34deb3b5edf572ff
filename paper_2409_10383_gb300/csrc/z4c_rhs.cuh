// Device-side finite differences and the Z4c right-hand side at one cell.
//
// Paper Sec. 2: vacuum Z4c with Bona-Masso lapse and Gamma-driver shift (the
// continuum equations are those of GR-Athena++, which the paper adopts
// unchanged); Sec. 3.2: cell-centred finite differences; Sec. 4.3:
// Kreiss-Oliger dissipation and kappa1/kappa2 constraint damping.
//
// Templated on the differencing order (4 or 6) and on the arithmetic type R
// of the stencils and algebra (double, or float for the FP32-RHS variant).
// Every stencil is evaluated as a sum over symmetric / antisymmetric pairs
// with small integer weights (exact in either precision), followed by one
// multiply with a per-block scale 1/(denominator h^p): this is the fewest
// FP64 operations per derivative on a part whose FP64 pipe is the bound.
#pragma once

#include <type_traits>

#include "z4c_internal.cuh"

namespace z4c {

template <class R>
__device__ __forceinline__ R ldg_(const R *p) {
  return __ldg(p);
}

// Stencil source: field f of the centre cell is at base[f * S].  Offsets
// are in elements.  The FP32 shadow stores chi, the gt diagonal and alpha
// minus one (shadow_shifted), so centre values add it back.
template <class R, bool SHIFTED_DIAG>
struct Src {
  const R *__restrict__ base;  // field 0 of the block (the same for the whole CTA)
  int32_t c;                   // storage index of the centre cell
  int32_t S;                   // cells per field
  __device__ __forceinline__ R at(int f, int off) const { return ldg_(base + (c + (f * S + off))); }
  __device__ __forceinline__ R val(int f) const {
    R v = at(f, 0);
    if (SHIFTED_DIAG && shadow_shifted(f)) v += R(1);
    return v;
  }
};

template <int ORD>
struct FD;

// 2nd order (2 ghosts): d1 = (f1 - f-1) / 2h, d2 = (f1 + f-1 - 2 f0) / h^2
//            (lopsided advection and KO dissipation: KoAdv<2> below)
template <>
struct FD<2> {
  static constexpr int W = 1;
  template <class S_>
  __device__ static auto d1(const S_ &s, int f, int st) {
    return s.at(f, st) - s.at(f, -st);
  }
  template <class S_>
  __device__ static auto d2(const S_ &s, int f, int st) {
    auto c = s.at(f, 0);
    auto a = s.at(f, st) + s.at(f, -st);
    return fma(c, decltype(c)(-2), a);
  }
  template <class S_>
  __device__ static auto mix(const S_ &s, int f, int sa, int sb) {
    return (s.at(f, sa + sb) - s.at(f, -sa + sb)) - (s.at(f, sa - sb) - s.at(f, -sa - sb));
  }
};

// 4th order: d1 = (8 (f1 - f-1) - (f2 - f-2)) / 12h
//            d2 = (16 (f1 + f-1) - (f2 + f-2) - 30 f0) / 12h^2
//            (lopsided advection and KO dissipation: KoAdv<4> below)
template <>
struct FD<4> {
  static constexpr int W = 2;
  template <class S_>
  __device__ static auto d1(const S_ &s, int f, int st) {
    auto a = s.at(f, st) - s.at(f, -st);
    auto b = s.at(f, 2 * st) - s.at(f, -2 * st);
    return fma(a, decltype(a)(8), -b);
  }
  template <class S_>
  __device__ static auto d2(const S_ &s, int f, int st) {
    auto c = s.at(f, 0);
    auto a = s.at(f, st) + s.at(f, -st);
    auto b = s.at(f, 2 * st) + s.at(f, -2 * st);
    return fma(a, decltype(a)(16), fma(c, decltype(c)(-30), -b));
  }
  template <class S_>
  __device__ static auto mix(const S_ &s, int f, int sa, int sb) {
    // sum_{a,b=1..2} c_a c_b [(f(a,b) - f(-a,b)) - (f(a,-b) - f(-a,-b))], c = (8, -1)
    auto q = [&](int a, int b) {
      return (s.at(f, a * sa + b * sb) - s.at(f, -a * sa + b * sb)) -
             (s.at(f, a * sa - b * sb) - s.at(f, -a * sa - b * sb));
    };
    auto q11 = q(1, 1), q12 = q(1, 2), q21 = q(2, 1), q22 = q(2, 2);
    using R = decltype(q11);
    return fma(q11, R(64), fma(q12 + q21, R(-8), q22));
  }
};

// 6th order: d1 = (45 (f1 - f-1) - 9 (f2 - f-2) + (f3 - f-3)) / 60h
//            d2 = (270 (f1 + f-1) - 27 (f2 + f-2) + 2 (f3 + f-3) - 490 f0) / 180h^2
//            (lopsided advection and KO dissipation: KoAdv<6> below)
template <>
struct FD<6> {
  static constexpr int W = 3;
  template <class S_>
  __device__ static auto d1(const S_ &s, int f, int st) {
    auto a = s.at(f, st) - s.at(f, -st);
    auto b = s.at(f, 2 * st) - s.at(f, -2 * st);
    auto c = s.at(f, 3 * st) - s.at(f, -3 * st);
    using R = decltype(a);
    return fma(a, R(45), fma(b, R(-9), c));
  }
  template <class S_>
  __device__ static auto d2(const S_ &s, int f, int st) {
    auto c0 = s.at(f, 0);
    auto a = s.at(f, st) + s.at(f, -st);
    auto b = s.at(f, 2 * st) + s.at(f, -2 * st);
    auto c = s.at(f, 3 * st) + s.at(f, -3 * st);
    using R = decltype(a);
    return fma(a, R(270), fma(b, R(-27), fma(c, R(2), c0 * R(-490))));
  }
  template <class S_>
  __device__ static auto mix(const S_ &s, int f, int sa, int sb) {
    auto q = [&](int a, int b) {
      return (s.at(f, a * sa + b * sb) - s.at(f, -a * sa + b * sb)) -
             (s.at(f, a * sa - b * sb) - s.at(f, -a * sa - b * sb));
    };
    auto q11 = q(1, 1), q12 = q(1, 2), q13 = q(1, 3);
    auto q21 = q(2, 1), q22 = q(2, 2), q23 = q(2, 3);
    auto q31 = q(3, 1), q32 = q(3, 2), q33 = q(3, 3);
    using R = decltype(q11);
    // c = (45, -9, 1): weights c_a c_b
    R r = q11 * R(2025);
    r = fma(q12 + q21, R(-405), r);
    r = fma(q13 + q31, R(45), r);
    r = fma(q22, R(81), r);
    r = fma(q23 + q32, R(-9), r);
    return r + q33;
  }
};

// Kreiss-Oliger dissipation (all three directions) plus lopsided advection
// beta^k d_k f of one field over its 3 x (2KW+1)-point cross: the lopsided
// stencil takes its points from the same cross, mirrored when beta^k < 0
// (the mirror image of the beta > 0 stencil).  lop() and ko() evaluate them
// from loaded points (unscaled: times slop |beta^k| and sko by the caller);
// kcoef()/lcoef() give the same coefficients for KoAdvWeights below.
template <int ORD>
struct KoAdv;
template <>
struct KoAdv<2> {
  // lopsided (beta > 0) offsets 0..2: (-3, 4, -1) / 2h;
  // KO: N = 2, (-1) sigma / (16 h) * (1 -4 6 -4 1) per direction
  static constexpr int KW = 2;
  static constexpr int LOFF = 0, LN = 3;
  template <class R>
  __device__ static R lop(const R *v) {
    return fma(v[0], R(-3), fma(v[1], R(4), -v[2]));
  }
  template <class R>
  __device__ static R ko(R c, const R *p) {
    return fma(c, R(18), fma(p[0], R(-4), p[1]));
  }
  __host__ __device__ static constexpr int kcoef(int m) { return m == 0 ? 6 : m == 1 ? -4 : 1; }
  __host__ __device__ static constexpr int lcoef(int m) { return m == 0 ? -3 : m == 1 ? 4 : m == 2 ? -1 : 0; }
};
template <>
struct KoAdv<4> {
  // lopsided (beta > 0) offsets -1..3: (-3, -10, 18, -6, 1) / 12h;
  // KO: N = 3, (+1) sigma / (64 h) * (1 -6 15 -20 15 -6 1) per direction
  static constexpr int KW = 3;                       // KO half width (N = 3)
  static constexpr int LOFF = -1, LN = 5;            // lopsided offsets -1..3
  template <class R>
  __device__ static R lop(const R *v) {              // v[m - LOFF] = f(m) upwind-oriented
    return fma(v[0], R(-3), fma(v[1], R(-10), fma(v[2], R(18), fma(v[3], R(-6), v[4]))));
  }
  template <class R>
  __device__ static R ko(R c, const R *p) {          // p[m-1] = sum over directions of f(+m) + f(-m)
    return fma(c, R(-60), fma(p[0], R(15), fma(p[1], R(-6), p[2])));
  }
  // per-direction KO coefficient of f(+-m) and lopsided coefficient of f(m)
  // (beta > 0 orientation; zero outside -1..3), in units of sko and slop
  __host__ __device__ static constexpr int kcoef(int m) {
    return m == 0 ? -20 : m == 1 ? 15 : m == 2 ? -6 : 1;
  }
  __host__ __device__ static constexpr int lcoef(int m) {
    return m == -1 ? -3 : m == 0 ? -10 : m == 1 ? 18 : m == 2 ? -6 : m == 3 ? 1 : 0;
  }
};
template <>
struct KoAdv<6> {
  // lopsided (beta > 0) offsets -2..4: (2, -24, -35, 80, -30, 8, -1) / 60h;
  // KO: N = 4, (-1) sigma / (256 h) * (1 -8 28 -56 70 -56 28 -8 1) per direction
  static constexpr int KW = 4;
  static constexpr int LOFF = -2, LN = 7;            // lopsided offsets -2..4
  template <class R>
  __device__ static R lop(const R *v) {
    return fma(v[0], R(2), fma(v[1], R(-24), fma(v[2], R(-35), fma(v[3], R(80),
               fma(v[4], R(-30), fma(v[5], R(8), -v[6]))))));
  }
  template <class R>
  __device__ static R ko(R c, const R *p) {
    return fma(c, R(210), fma(p[0], R(-56), fma(p[1], R(28), fma(p[2], R(-8), p[3]))));
  }
  __host__ __device__ static constexpr int kcoef(int m) {
    return m == 0 ? 70 : m == 1 ? -56 : m == 2 ? 28 : m == 3 ? -8 : 1;
  }
  __host__ __device__ static constexpr int lcoef(int m) {
    return m == -2 ? 2 : m == -1 ? -24 : m == 0 ? -35 : m == 1 ? 80 : m == 2 ? -30 : m == 3 ? 8
                       : m == 4 ? -1 : 0;
  }
};

// The same two operators as one stencil per direction.  KO and the lopsided
// derivative act on the same points of each field, and their coefficients
// depend on the cell (sko, |beta^d| slop, the sign of beta^d) but not on the
// field: w[d][.] holds, per direction d, the coefficient of f(m st_d) in
// sko KO_d + |beta^d| slop Lop_d for m = -W..-1 (index m + W) and m = 1..W
// (index m + W - 1), the lopsided stencil mirrored for beta^d < 0; w0 is the
// centre coefficient summed over the three directions.  Formed once per
// cell, then each field costs 2W DFMA per direction instead of the pair sums,
// the lopsided sums and the per-point orientation selects of ko_adv.
template <int ORD, class R>
struct KoAdvWeights {
  static constexpr int W = KoAdv<ORD>::KW;
  R w[3][2 * W];
  R w0;
  __device__ __forceinline__ KoAdvWeights(const bool up[3], const R ab[3], R sko) {
    using K = KoAdv<ORD>;
    R kw[W + 1];
#pragma unroll
    for (int m = 0; m <= W; ++m) kw[m] = sko * R(K::kcoef(m));
    w0 = fma(ab[0] + ab[1] + ab[2], R(K::lcoef(0)), R(3) * kw[0]);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int m = 1; m <= W; ++m) {
        const R lp = R(K::lcoef(m)), lm = R(K::lcoef(-m));
        w[d][W + m - 1] = fma(ab[d], up[d] ? lp : lm, kw[m]);
        w[d][W - m] = fma(ab[d], up[d] ? lm : lp, kw[m]);
      }
    }
  }
  // acc + (KO + advection) of field f: one accumulation chain per direction
  template <class S_>
  __device__ __forceinline__ R apply(const S_ &s, int f, const int st[3], R acc) const {
    R a[3];
    a[0] = fma(w0, s.at(f, 0), acc);
    a[1] = w[1][0] * s.at(f, -W * st[1]);
    a[2] = w[2][0] * s.at(f, -W * st[2]);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int m = -W; m <= W; ++m) {
        if (m == 0 || (d > 0 && m == -W)) continue;
        a[d] = fma(w[d][m < 0 ? m + W : m + W - 1], s.at(f, m * st[d]), a[d]);
      }
    }
    return a[0] + (a[1] + a[2]);
  }
  // The same sum written with the centre subtracted,
  // sum_{d, m != 0} w[d][m] (f(m st_d) - f(0)): both stencils annihilate
  // constants, so the centre coefficient drops out and a field that is
  // constant along a direction contributes exactly zero there.  Used in FP32,
  // where the rounded weights would otherwise leave a residue of
  // eps |f| sko per direction (the FP32 pipe has the slack for the
  // subtractions; the FP64 path, bound by its pipe, takes apply()).
  template <class S_>
  __device__ __forceinline__ R apply_diff(const S_ &s, int f, const int st[3]) const {
    const R c = s.at(f, 0);
    R a[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      a[d] = w[d][0] * (s.at(f, -W * st[d]) - c);
#pragma unroll
      for (int m = -W + 1; m <= W; ++m) {
        if (m == 0) continue;
        a[d] = fma(w[d][m < 0 ? m + W : m + W - 1], s.at(f, m * st[d]) - c, a[d]);
      }
    }
    return a[0] + (a[1] + a[2]);
  }
};

// ---- two cells per thread: FP32 pairs on the packed f32x2 instructions ----
//
// F2 holds the same quantity at two neighbouring cells (x and x + 1).  Its
// arithmetic issues one packed instruction (add / sub / mul / fma .f32x2)
// for both cells.  A product is kept unevaluated (F2Mul) until it meets an
// addition, which then becomes one fused multiply-add, so a * b + c costs
// one instruction as it does for a scalar float.  Each lane rounds like the
// scalar FP32 path; where the two fuse differently the results differ by
// FP32 rounding only.
using ::fabs;  // the scalar overloads stay visible beside the F2 ones below
using ::fma;
struct F2 {
  float2 v;
  F2() = default;
  __device__ __forceinline__ F2(float2 a) : v(a) {}
  __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
  template <class T, class = typename std::enable_if<std::is_arithmetic<T>::value>::type>
  __device__ __forceinline__ explicit F2(T x) : v(make_float2(float(x), float(x))) {}
};
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long *>(&a)), "l"(*reinterpret_cast<unsigned long long *>(&b)));
  return *reinterpret_cast<float2 *>(&d);
}
struct F2Mul {
  F2 a, b;
  __device__ __forceinline__ operator F2() const { return F2(__fmul2_rn(a.v, b.v)); }
};
__device__ __forceinline__ F2 fma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2Mul operator*(F2 a, F2 b) { return F2Mul{a, b}; }
__device__ __forceinline__ F2Mul operator*(F2Mul m, F2 b) { return F2Mul{F2(m), b}; }
__device__ __forceinline__ F2Mul operator*(F2 a, F2Mul m) { return F2Mul{a, F2(m)}; }
__device__ __forceinline__ F2Mul operator*(F2Mul m, F2Mul n) { return F2Mul{F2(m), F2(n)}; }
__device__ __forceinline__ F2Mul operator-(F2Mul m) { return F2Mul{-m.a, m.b}; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(f2_sub(a.v, b.v)); }
__device__ __forceinline__ F2 operator+(F2Mul m, F2 c) { return fma(m.a, m.b, c); }
__device__ __forceinline__ F2 operator+(F2 c, F2Mul m) { return fma(m.a, m.b, c); }
__device__ __forceinline__ F2 operator-(F2 c, F2Mul m) { return fma(-m.a, m.b, c); }
__device__ __forceinline__ F2 operator-(F2Mul m, F2 c) { return fma(m.a, m.b, -c); }
__device__ __forceinline__ F2 operator+(F2Mul m, F2Mul n) { return fma(m.a, m.b, F2(n)); }
__device__ __forceinline__ F2 operator-(F2Mul m, F2Mul n) { return fma(m.a, m.b, -F2(n)); }
__device__ __forceinline__ F2 operator/(F2 a, F2 b) { return F2(a.v.x / b.v.x, a.v.y / b.v.y); }
__device__ __forceinline__ F2 &operator+=(F2 &a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2 &operator+=(F2 &a, F2Mul m) { return a = a + m; }
__device__ __forceinline__ F2 &operator-=(F2 &a, F2 b) { return a = a - b; }
__device__ __forceinline__ F2 &operator-=(F2 &a, F2Mul m) { return a = a - m; }
__device__ __forceinline__ F2 fabs(F2 a) { return F2(fabsf(a.v.x), fabsf(a.v.y)); }
template <class R>
struct is_pair : std::false_type {};
template <>
struct is_pair<F2> : std::true_type {};

// Stencil source for a cell pair: field f of the even cell c (and c + 1) of
// an FP32 array whose row starts are 8-byte aligned (every storage extent
// and block offset even).  An even offset is one aligned 8-byte load; an odd
// offset takes the upper half of the pair below and the lower half of the
// pair above.  SHIFTED: the FP32 shadow's shadow_shifted fields are stored
// minus one.
template <bool SHIFTED>
struct SrcPair {
  const float *__restrict__ base;
  int32_t c;
  int32_t S;
  __device__ __forceinline__ F2 at(int f, int off) const {
    const float *p = base + (c + (f * S + off));
    if ((off & 1) == 0) return F2(__ldg(reinterpret_cast<const float2 *>(p)));
    const float2 lo = __ldg(reinterpret_cast<const float2 *>(p - 1));
    const float2 hi = __ldg(reinterpret_cast<const float2 *>(p + 1));
    return F2(lo.y, hi.x);
  }
  __device__ __forceinline__ F2 val(int f) const {
    F2 v = at(f, 0);
    if (SHIFTED && shadow_shifted(f)) v += F2(1.0f);
    return v;
  }
};

// KO dissipation + lopsided advection for a cell pair: per lane the same
// per-cell weights as KoAdvWeights (oriented by the sign of beta^d at that
// cell), applied to the differences f(m st_d) - f(0) as in apply_diff.
template <int ORD>
struct KoAdvWeightsPair {
  static constexpr int W = KoAdv<ORD>::KW;
  F2 w[3][2 * W];
  __device__ __forceinline__ KoAdvWeightsPair(const F2 beta[3], float slop, float sko) {
    using K = KoAdv<ORD>;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float b0 = beta[d].v.x, b1 = beta[d].v.y;
      const bool up0 = b0 >= 0.f, up1 = b1 >= 0.f;
      const float ab0 = fabsf(b0) * slop, ab1 = fabsf(b1) * slop;
#pragma unroll
      for (int m = 1; m <= W; ++m) {
        const float kw = sko * float(K::kcoef(m));
        const float lp = float(K::lcoef(m)), lm = float(K::lcoef(-m));
        w[d][W + m - 1] = F2(fmaf(ab0, up0 ? lp : lm, kw), fmaf(ab1, up1 ? lp : lm, kw));
        w[d][W - m] = F2(fmaf(ab0, up0 ? lm : lp, kw), fmaf(ab1, up1 ? lm : lp, kw));
      }
    }
  }
  template <class S_>
  __device__ __forceinline__ F2 apply_diff(const S_ &s, int f, const int st[3]) const {
    const F2 c = s.at(f, 0);
    F2 a[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      a[d] = w[d][0] * (s.at(f, -W * st[d]) - c);
#pragma unroll
      for (int m = -W + 1; m <= W; ++m) {
        if (m == 0) continue;
        a[d] = fma(w[d][m < 0 ? m + W : m + W - 1], s.at(f, m * st[d]) - c, a[d]);
      }
    }
    return a[0] + (a[1] + a[2]);
  }
};

// Scale factors of one block in precision R.
template <class R>
struct Scales {
  R s1, s2, smix, slop, sko;
};
__device__ __forceinline__ Scales<double> scales_of(const DevBlock &b, double) {
  return {b.s1, b.s2, b.smix, b.slop, b.sko};
}
__device__ __forceinline__ Scales<float> scales_of(const DevBlock &b, float) {
  return {b.s1f, b.s2f, b.smixf, b.slopf, b.skof};
}

template <class R>
struct Phys {
  R kappa1, kappa2, eta;
  int lapse, shift;
};

// Derivative providers.  Direct evaluates every stencil from the state;
// Pre takes the y and z first derivatives of the eleven fields that also
// need mixed second derivatives (chi, gt_ij, alpha, beta^i) from arrays
// filled by a preceding pass, so that d_x d_y f = D_x (D_y f),
// d_x d_z f = D_x (D_z f) and d_y d_z f = D_y (D_z f) are one first-derivative
// stencil each (the tensor-product definition, evaluated in two passes).
template <int ORD, class R, class SRC>
struct Direct {
  static constexpr bool kStagedKO = false;  // KO / advection evaluated from s by KoAdvWeights
  const SRC &s;
  const int *st;
  Scales<R> sc;
  __device__ __forceinline__ R d1(int f, int d) const { return FD<ORD>::d1(s, f, st[d]) * sc.s1; }
  __device__ __forceinline__ R d2(int f, int d) const { return FD<ORD>::d2(s, f, st[d]) * sc.s2; }
  __device__ __forceinline__ R mix(int f, int a, int b) const {
    return FD<ORD>::mix(s, f, st[a], st[b]) * sc.smix;
  }
  // the same before the scale, and the scales (d2 = d2raw * d2scale, ...)
  __device__ __forceinline__ R d2raw(int f, int d) const { return FD<ORD>::d2(s, f, st[d]); }
  __device__ __forceinline__ R mixraw(int f, int a, int b) const { return FD<ORD>::mix(s, f, st[a], st[b]); }
  __device__ __forceinline__ R d2scale() const { return sc.s2; }
  __device__ __forceinline__ R mixscale() const { return sc.smix; }
};

// slot of a field in the stored-derivative arrays (-1: not stored);
// arrays 0..10 hold D_y f, arrays 11..21 hold D_z f
__host__ __device__ constexpr int dslot(int f) {
  return f == CHI ? 0 : (f >= GXX && f <= GZZ) ? f - GXX + 1 : f == ALPHA ? 7 : (f >= BETAX) ? f - BETAX + 8 : -1;
}

template <int ORD, class R, class SRC, class DS>
struct Pre {
  static constexpr bool kStagedKO = false;
  const SRC &s;
  const DS &ds;  // stored derivatives at this cell (already multiplied by s1)
  const int *st;
  Scales<R> sc;
  __device__ __forceinline__ R d1(int f, int d) const {
    const int q = dslot(f);
    if (d > 0 && q >= 0) return ds.at(q + (d - 1) * NDS, 0);
    return FD<ORD>::d1(s, f, st[d]) * sc.s1;
  }
  __device__ __forceinline__ R d2(int f, int d) const { return FD<ORD>::d2(s, f, st[d]) * sc.s2; }
  __device__ __forceinline__ R mix(int f, int a, int b) const {
    const int q = dslot(f);
    if (a == 0 && b == 1) return FD<ORD>::d1(ds, q, st[0]) * sc.s1;         // D_x (D_y f)
    if (a == 0 && b == 2) return FD<ORD>::d1(ds, q + NDS, st[0]) * sc.s1;   // D_x (D_z f)
    return FD<ORD>::d1(ds, q + NDS, st[1]) * sc.s1;                         // D_y (D_z f)
  }
  __device__ __forceinline__ R d2raw(int f, int d) const { return FD<ORD>::d2(s, f, st[d]); }
  __device__ __forceinline__ R mixraw(int f, int a, int b) const {
    const int q = dslot(f);
    if (a == 0 && b == 1) return FD<ORD>::d1(ds, q, st[0]);
    if (a == 0 && b == 2) return FD<ORD>::d1(ds, q + NDS, st[0]);
    return FD<ORD>::d1(ds, q + NDS, st[1]);
  }
  __device__ __forceinline__ R d2scale() const { return sc.s2; }
  __device__ __forceinline__ R mixscale() const { return sc.s1; }
};

template <class R>
__device__ __forceinline__ R trsym(const R gi[6], const R X[6]) {  // gt^ij X_ij
  return gi[0] * X[0] + gi[3] * X[3] + gi[5] * X[5] + R(2) * (gi[1] * X[1] + gi[2] * X[2] + gi[4] * X[4]);
}
template <class R>
__device__ __forceinline__ R quad(const R gi[6], const R a[3], const R b[3]) {  // gt^lm a_l b_m
  return gi[0] * a[0] * b[0] + gi[3] * a[1] * b[1] + gi[5] * a[2] * b[2] +
         gi[1] * (a[0] * b[1] + a[1] * b[0]) + gi[2] * (a[0] * b[2] + a[2] * b[0]) +
         gi[4] * (a[1] * b[2] + a[2] * b[1]);
}

// gt^ij = adj(gt) / det(gt)
template <class R>
__device__ __forceinline__ void inverse_metric(const R g[6], R gi[6]) {
  R axx = g[3] * g[5] - g[4] * g[4];
  R axy = g[2] * g[4] - g[1] * g[5];
  R axz = g[1] * g[4] - g[2] * g[3];
  R ayy = g[0] * g[5] - g[2] * g[2];
  R ayz = g[1] * g[2] - g[0] * g[4];
  R azz = g[0] * g[3] - g[1] * g[1];
  R idet = R(1) / (g[0] * axx + g[1] * axy + g[2] * axz);
  gi[0] = axx * idet; gi[1] = axy * idet; gi[2] = axz * idet;
  gi[3] = ayy * idet; gi[4] = ayz * idet; gi[5] = azz * idet;
}

// Gl[i][jk] = Gt_ijk = (d_j gt_ik + d_k gt_ij - d_i gt_jk)/2, Gu[i][jk] = Gt^i_jk,
// Gd^i = gt^jk Gt^i_jk.  dg[d][q] = d_d gt_q.
template <class R>
__device__ __forceinline__ void christoffel(const R gi[6], const R dg[3][6], R Gl[3][6], R Gu[3][6],
                                            R Gd[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k2 = j; k2 < 3; ++k2)
        Gl[i][S6(j, k2)] = R(0.5) * (dg[j][S6(i, k2)] + dg[k2][S6(i, j)] - dg[i][S6(j, k2)]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int q = 0; q < 6; ++q)
      Gu[i][q] = gi[S6(i, 0)] * Gl[0][q] + gi[S6(i, 1)] * Gl[1][q] + gi[S6(i, 2)] * Gl[2][q];
#pragma unroll
  for (int i = 0; i < 3; ++i) Gd[i] = trsym(gi, Gu[i]);
}

// Ricci tensor R_ij = Rt_ij + Rchi_ij of the physical metric gt_ij / chi:
//   Rt_ij   = -1/2 gt^lm d_l d_m gt_ij + gt_k(i d_j) Gam^k + Gd^k Gt_(ij)k
//             + gt^lm (2 Gt^k_l(i Gt_j)km + Gt^k_im Gt_klj)
//   Rchi_ij = (DDchi_ij + gt_ij gt^lm DDchi_lm) / (2 chi)
//             - (d_i chi d_j chi + 3 gt_ij gt^lm d_l chi d_m chi) / (4 chi^2)
// with DDchi_ij = d_i d_j chi - Gt^k_ij d_k chi and 1/chi -> ichi.
// The quadratic Christoffel terms are summed as
//   sum_km U[k][m][i] d_m gt_jk + U[k][m][j] Gt_ikm,  U[k][m][i] = gt^lm Gt^k_li:
// the term gt^lm Gt^k_im Gt_klj equals sum_km U[k][m][i] Gt_kmj, and
// Gt_jkm + Gt_kmj = d_m gt_jk by the definition of Gt_ijk, so two of the
// three contractions collapse into one against the metric derivatives.
template <class R, class DV>
__device__ __forceinline__ void ricci(const DV &dv, R ichi,
                                      const R g[6], const R gi[6], const R dchi[3], const R dg[3][6],
                                      const R dGam[3][3], const R Gl[3][6], const R Gu[3][6],
                                      const R Gd[3], const R DDchi[6], R Ric[6]) {
  // U[k][m][i] = gt^lm Gt^k_li
  R U[3][3][3];
#pragma unroll
  for (int k2 = 0; k2 < 3; ++k2)
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        U[k2][m][i] = gi[S6(0, m)] * Gu[k2][S6(0, i)] + gi[S6(1, m)] * Gu[k2][S6(1, i)] +
                      gi[S6(2, m)] * Gu[k2][S6(2, i)];
  const R trDDchi = trsym(gi, DDchi);
  const R dchi2 = quad(gi, dchi, dchi);
  // -1/2 gt^lm d_l d_m gt_ij.  Scalar types: the stencils' scales and the
  // factors -1/2 (diagonal) and -1 (off-diagonal pairs) are folded into
  // gt^lm once per cell, so the 36 second derivatives of gt are taken
  // unscaled (42 fewer multiplies per cell).  Cell pairs keep the scaled
  // form: the six folded weights would cost them registers they lack.
  constexpr bool fold = !is_pair<R>::value;
  R gs[6];
  if constexpr (fold) {
    const R cd = R(-0.5) * dv.d2scale(), cm = -dv.mixscale();
    gs[0] = cd * gi[0]; gs[1] = cm * gi[1]; gs[2] = cm * gi[2];
    gs[3] = cd * gi[3]; gs[4] = cm * gi[4]; gs[5] = cd * gi[5];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int q = S6(i, j);
      R r;
      if constexpr (fold) {
        r = gs[0] * dv.d2raw(GXX + q, 0) + gs[3] * dv.d2raw(GXX + q, 1) + gs[5] * dv.d2raw(GXX + q, 2);
        r += gs[1] * dv.mixraw(GXX + q, 0, 1) + gs[2] * dv.mixraw(GXX + q, 0, 2) + gs[4] * dv.mixraw(GXX + q, 1, 2);
      } else {
        R dd[6];
        dd[0] = dv.d2(GXX + q, 0);
        dd[3] = dv.d2(GXX + q, 1);
        dd[5] = dv.d2(GXX + q, 2);
        dd[1] = dv.mix(GXX + q, 0, 1);
        dd[2] = dv.mix(GXX + q, 0, 2);
        dd[4] = dv.mix(GXX + q, 1, 2);
        r = R(-0.5) * trsym(gi, dd);
      }
      R t = R(0);
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) t += g[S6(k2, i)] * dGam[j][k2] + g[S6(k2, j)] * dGam[i][k2];
      r += R(0.5) * t;
      t = R(0);
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) t += Gd[k2] * (Gl[i][S6(j, k2)] + Gl[j][S6(i, k2)]);
      r += R(0.5) * t;
      t = R(0);
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2)
#pragma unroll
        for (int m = 0; m < 3; ++m) t += U[k2][m][i] * dg[m][S6(j, k2)] + U[k2][m][j] * Gl[i][S6(k2, m)];
      r += t;
      R rc = R(0.5) * ichi * (DDchi[q] + g[q] * trDDchi) -
             R(0.25) * ichi * ichi * (dchi[i] * dchi[j] + R(3) * g[q] * dchi2);
      Ric[q] = r + rc;
    }
}

// Z4c right-hand side at one interior cell.  ichi = 1 / max(chi, chi_floor)
// (computed by the caller in FP64).  st = element strides (1, e0, e0 e1).
template <int ORD, class R, class SRC, class DV>
__device__ __forceinline__ void rhs_point(const SRC &s, const DV &dv, const int st[3], const Scales<R> &sc,
                                          const Phys<R> &p, R ichi, R k[NF]) {
  using F = FD<ORD>;
  const R chi = s.val(CHI), Khat = s.val(KHAT), Theta = s.val(THETA), al = s.val(ALPHA);
  R g[6], A[6], Gam[3], beta[3];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    g[q] = s.val(GXX + q);
    A[q] = s.val(AXX + q);
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Gam[i] = s.val(GAMX + i);
    beta[i] = s.val(BETAX + i);
  }
  R gi[6];
  inverse_metric(g, gi);

  // first derivatives
  R dchi[3], dal[3], dKhat[3], dTheta[3], dbeta[3][3], dGam[3][3], dg[3][6];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dchi[d] = dv.d1(CHI, d);
    dal[d] = dv.d1(ALPHA, d);
    dKhat[d] = dv.d1(KHAT, d);
    dTheta[d] = dv.d1(THETA, d);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dbeta[d][i] = dv.d1(BETAX + i, d);
      dGam[d][i] = dv.d1(GAMX + i, d);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) dg[d][q] = dv.d1(GXX + q, d);
  }

  R Gl[3][6], Gu[3][6], Gd[3];
  christoffel(gi, dg, Gl, Gu, Gd);

  // second derivatives of chi and alpha, covariant parts
  R DDchi[6], DDa0[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int q = S6(i, j);
      R ddc, dda;
      if (i == j) {
        ddc = dv.d2(CHI, i);
        dda = dv.d2(ALPHA, i);
      } else {
        ddc = dv.mix(CHI, i, j);
        dda = dv.mix(ALPHA, i, j);
      }
      DDchi[q] = ddc - (Gu[0][q] * dchi[0] + Gu[1][q] * dchi[1] + Gu[2][q] * dchi[2]);
      DDa0[q] = dda - (Gu[0][q] * dal[0] + Gu[1][q] * dal[1] + Gu[2][q] * dal[2]);
    }
  auto trsym = [&](const R *X) { return z4c::trsym(gi, X); };
  auto quad = [&](const R *a, const R *b) { return z4c::quad(gi, a, b); };

  R Ric[6];
  ricci(dv, ichi, g, gi, dchi, dg, dGam, Gl, Gu, Gd, DDchi, Ric);
  const R Rs = chi * trsym(Ric);

  // D_i D_j alpha and its trace
  const R dchi_dal = quad(dchi, dal);
  R DDa[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int q = S6(i, j);
      DDa[q] = DDa0[q] + R(0.5) * ichi * (dchi[i] * dal[j] + dchi[j] * dal[i] - g[q] * dchi_dal);
    }
  const R lapl_a = chi * trsym(DDa0) - R(0.5) * dchi_dal;

  // At^ij, At_ij At^ij, At_ik gt^kl At_lj
  R M[3][3];  // M[i][l] = gt^ik At_kl
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int l = 0; l < 3; ++l)
      M[i][l] = gi[S6(i, 0)] * A[S6(0, l)] + gi[S6(i, 1)] * A[S6(1, l)] + gi[S6(i, 2)] * A[S6(2, l)];
  R Au[6], AA2[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int q = S6(i, j);
      Au[q] = M[i][0] * gi[S6(0, j)] + M[i][1] * gi[S6(1, j)] + M[i][2] * gi[S6(2, j)];
      AA2[q] = M[0][i] * A[S6(0, j)] + M[1][i] * A[S6(1, j)] + M[2][i] * A[S6(2, j)];
    }
  const R AA = A[0] * Au[0] + A[3] * Au[3] + A[5] * Au[5] + R(2) * (A[1] * Au[1] + A[2] * Au[2] + A[4] * Au[4]);

  const R K = Khat + R(2) * Theta;
  const R divb = dbeta[0][0] + dbeta[1][1] + dbeta[2][2];
  const R two3 = R(2) / R(3), third = R(1) / R(3);

  k[CHI] = two3 * chi * (al * K - divb);

#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int q = S6(i, j);
      R t = R(-2) * al * A[q] - two3 * g[q] * divb;
#pragma unroll
      for (int k2 = 0; k2 < 3; ++k2) t += g[S6(i, k2)] * dbeta[j][k2] + g[S6(j, k2)] * dbeta[i][k2];
      k[GXX + q] = t;
    }

  k[KHAT] = -lapl_a + al * (AA + third * K * K) + p.kappa1 * (R(1) - p.kappa2) * al * Theta;

  {
    R X[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) X[q] = al * Ric[q] - DDa[q];
    const R trX = trsym(X);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int q = S6(i, j);
        R t = chi * (X[q] - third * g[q] * trX) + al * (K * A[q] - R(2) * AA2[q]) - two3 * A[q] * divb;
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) t += A[S6(i, k2)] * dbeta[j][k2] + A[S6(j, k2)] * dbeta[i][k2];
        k[AXX + q] = t;
      }
  }

  k[THETA] = R(0.5) * al * (Rs - AA + two3 * K * K) - al * p.kappa1 * (R(2) + p.kappa2) * Theta;

  {
    // d_j d_k beta^i, and d_j (d_k beta^k).  Scalar types: the second
    // derivatives are taken unscaled, the stencil scales (and the factor 2
    // of the off-diagonal pairs) folded into gt^jk once per cell, as for
    // the Ricci tensor; cell pairs keep the scaled form.
    constexpr bool foldb = !is_pair<R>::value;
    R ddb[3][6];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if constexpr (foldb) {
        ddb[i][0] = dv.d2raw(BETAX + i, 0);
        ddb[i][3] = dv.d2raw(BETAX + i, 1);
        ddb[i][5] = dv.d2raw(BETAX + i, 2);
        ddb[i][1] = dv.mixraw(BETAX + i, 0, 1);
        ddb[i][2] = dv.mixraw(BETAX + i, 0, 2);
        ddb[i][4] = dv.mixraw(BETAX + i, 1, 2);
      } else {
        ddb[i][0] = dv.d2(BETAX + i, 0);
        ddb[i][3] = dv.d2(BETAX + i, 1);
        ddb[i][5] = dv.d2(BETAX + i, 2);
        ddb[i][1] = dv.mix(BETAX + i, 0, 1);
        ddb[i][2] = dv.mix(BETAX + i, 0, 2);
        ddb[i][4] = dv.mix(BETAX + i, 1, 2);
      }
    }
    R ddivb[3];
    R gw[6];
    if constexpr (foldb) {
      const R s2 = dv.d2scale(), sm = dv.mixscale(), sm2 = sm + sm;
      gw[0] = s2 * gi[0]; gw[1] = sm2 * gi[1]; gw[2] = sm2 * gi[2];
      gw[3] = s2 * gi[3]; gw[4] = sm2 * gi[4]; gw[5] = s2 * gi[5];
      ddivb[0] = fma(s2, ddb[0][0], sm * (ddb[1][1] + ddb[2][2]));
      ddivb[1] = fma(s2, ddb[1][3], sm * (ddb[0][1] + ddb[2][4]));
      ddivb[2] = fma(s2, ddb[2][5], sm * (ddb[0][2] + ddb[1][4]));
    } else {
#pragma unroll
      for (int j = 0; j < 3; ++j) ddivb[j] = ddb[0][S6(j, 0)] + ddb[1][S6(j, 1)] + ddb[2][S6(j, 2)];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      R t;
      if constexpr (foldb)
        t = gw[0] * ddb[i][0] + gw[3] * ddb[i][3] + gw[5] * ddb[i][5] + gw[1] * ddb[i][1] + gw[2] * ddb[i][2] +
            gw[4] * ddb[i][4];
      else
        t = trsym(ddb[i]);
      t += two3 * Gd[i] * divb;
      t -= Gd[0] * dbeta[0][i] + Gd[1] * dbeta[1][i] + Gd[2] * dbeta[2][i];
      R u = R(0), w = R(0), v = R(0), z = R(0);
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        u += Au[S6(i, j)] * dal[j];
        w += Au[S6(i, j)] * dchi[j];
        v += gi[S6(i, j)] * (R(2) * dKhat[j] + dTheta[j]);
        z += gi[S6(i, j)] * ddivb[j];
      }
      R GA = Gu[i][0] * Au[0] + Gu[i][3] * Au[3] + Gu[i][5] * Au[5] +
             R(2) * (Gu[i][1] * Au[1] + Gu[i][2] * Au[2] + Gu[i][4] * Au[4]);
      t += third * z - R(2) * u;
      t += R(2) * al * (GA - R(1.5) * ichi * w - third * v);
      t -= R(2) * al * p.kappa1 * (Gam[i] - Gd[i]);
      k[GAMX + i] = t;
    }
  }

  k[ALPHA] = p.lapse == 1 ? R(-2) * al * Khat : -al * al * Khat;
#pragma unroll
  for (int i = 0; i < 3; ++i) k[BETAX + i] = p.shift ? Gam[i] - p.eta * beta[i] : R(0);

  // lopsided advection along the shift and Kreiss-Oliger dissipation
  if constexpr (is_pair<R>::value) {
    // cell pairs: weights per lane; the result goes through a shared-memory
    // slot per field and thread as in the FP32 branch below
    const KoAdvWeightsPair<ORD> kaw(beta, sc.slop.v.x, sc.sko.v.x);
    __shared__ F2 kko2[NF][TX * TY / 2];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;  // 64 threads
#pragma unroll 2
    for (int f = 0; f < NF; ++f) kko2[f][tid] = (!p.shift && f >= BETAX) ? F2(0.0f) : kaw.apply_diff(s, f, st);
#pragma unroll
    for (int f = 0; f < NF; ++f) k[f] += kko2[f][tid];
  } else if constexpr (DV::kStagedKO) {
    // already evaluated per field by the staging pass
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      if (!p.shift && f >= BETAX) continue;
      k[f] += dv.ko(f);
    }
  } else {
    bool up[3];
    R ab[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      up[d] = beta[d] >= R(0);
      ab[d] = fabs(beta[d]) * sc.slop;
    }
    const KoAdvWeights<ORD, R> kaw(up, ab, sc.sko);
    // one field at a time (an unrolled loop exceeds the register budget)
    if constexpr (sizeof(R) == 4) {
      // FP32: the result goes to a shared-memory slot per field and cell, so
      // that k[] is only indexed by compile-time constants (a runtime index
      // into a register array costs a compare-and-select per element)
      __shared__ R kko[NF][TX * TY];
      const int tid = threadIdx.y * TX + threadIdx.x;
#pragma unroll 2
      for (int f = 0; f < NF; ++f)
        kko[f][tid] = (!p.shift && f >= BETAX) ? R(0) : kaw.apply_diff(s, f, st);
#pragma unroll
      for (int f = 0; f < NF; ++f) k[f] += kko[f][tid];
    } else {
      // FP64 (k[] lives in local memory here; the FP64 pipe is the bound)
#pragma unroll 1
      for (int f = 0; f < NF; ++f) {
        if (!p.shift && f >= BETAX) continue;
        k[f] = kaw.apply(s, f, st, k[f]);
      }
    }
  }
}

// Hamiltonian and momentum constraints at one interior cell (FP64):
//   H   = R + 2/3 K^2 - At_ij At^ij,   K = Khat + 2 Theta
//   M^i = d_j At^ij + Gt^i_jk At^jk - 3/2 At^ij d_j chi / chi - 2/3 gt^ij d_j K
// with d_j At^ij expanded by the product rule and
// d_k gt^ij = -gt^ia gt^jb d_k gt_ab.
template <int ORD, class SRC>
__device__ __forceinline__ void constraints_point(const SRC &s, const int st[3],
                                                  const Scales<double> &sc, double ichi,
                                                  double out[4]) {
  using F = FD<ORD>;
  using R = double;
  const R chi = s.val(CHI), K = s.val(KHAT) + 2.0 * s.val(THETA);
  R g[6], A[6], gi[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    g[q] = s.val(GXX + q);
    A[q] = s.val(AXX + q);
  }
  inverse_metric(g, gi);
  R dchi[3], dK[3], dGam[3][3], dg[3][6], dA[3][6];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dchi[d] = F::d1(s, CHI, st[d]) * sc.s1;
    dK[d] = (F::d1(s, KHAT, st[d]) + 2.0 * F::d1(s, THETA, st[d])) * sc.s1;
#pragma unroll
    for (int i = 0; i < 3; ++i) dGam[d][i] = F::d1(s, GAMX + i, st[d]) * sc.s1;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      dg[d][q] = F::d1(s, GXX + q, st[d]) * sc.s1;
      dA[d][q] = F::d1(s, AXX + q, st[d]) * sc.s1;
    }
  }
  R Gl[3][6], Gu[3][6], Gd[3];
  christoffel(gi, dg, Gl, Gu, Gd);
  R DDchi[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int q = S6(i, j);
      R ddc = i == j ? F::d2(s, CHI, st[i]) * sc.s2 : F::mix(s, CHI, st[i], st[j]) * sc.smix;
      DDchi[q] = ddc - (Gu[0][q] * dchi[0] + Gu[1][q] * dchi[1] + Gu[2][q] * dchi[2]);
    }
  R Ric[6];
  const Direct<ORD, double, SRC> dv{s, st, sc};
  ricci(dv, ichi, g, gi, dchi, dg, dGam, Gl, Gu, Gd, DDchi, Ric);
  // At^ij and At_ij At^ij
  R M[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int l = 0; l < 3; ++l)
      M[i][l] = gi[S6(i, 0)] * A[S6(0, l)] + gi[S6(i, 1)] * A[S6(1, l)] + gi[S6(i, 2)] * A[S6(2, l)];
  R Au[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j)
      Au[S6(i, j)] = M[i][0] * gi[S6(0, j)] + M[i][1] * gi[S6(1, j)] + M[i][2] * gi[S6(2, j)];
  const R AA = A[0] * Au[0] + A[3] * Au[3] + A[5] * Au[5] +
               2.0 * (A[1] * Au[1] + A[2] * Au[2] + A[4] * Au[4]);
  out[0] = chi * trsym(gi, Ric) + 2.0 / 3.0 * K * K - AA;
  // d_k gt^ij
  R dgi[3][6];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        R t = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) t += gi[S6(i, a)] * gi[S6(j, b)] * dg[d][S6(a, b)];
        dgi[d][S6(i, j)] = -t;
      }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R t = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          t += (dgi[j][S6(i, a)] * gi[S6(j, b)] + gi[S6(i, a)] * dgi[j][S6(j, b)]) * A[S6(a, b)] +
               gi[S6(i, a)] * gi[S6(j, b)] * dA[j][S6(a, b)];
    t += trsym(Au, Gu[i]);
#pragma unroll
    for (int j = 0; j < 3; ++j) t -= 1.5 * ichi * Au[S6(i, j)] * dchi[j] + 2.0 / 3.0 * gi[S6(i, j)] * dK[j];
    out[1 + i] = t;
  }
}

// Weyl scalar Psi4 at one interior cell (Sec. 3.3: the outgoing Weyl
// scalar in a coordinate tetrad), in FP64:
//   Psi4 = (E_ij - i B_ij) mb^i mb^j,
//   E_ij = R_ij + K K_ij - K_ik gamma^kl K_lj  (R_ij of gamma_ij = gt_ij / chi),
//   B_ij = sym(gamma_im C^m_j), C^m_j = [mkl] D_k K_lj / sqrt(det gamma),
//   K_ij = (At_ij + gt_ij K / 3) / chi, K = Khat + 2 Theta, its derivatives by
//   the product rule, D_k with the Christoffels of gamma,
//   G^m_kl = Gt^m_kl - (delta^m_k d_l chi + delta^m_l d_k chi
//            - gt_kl gt^mn d_n chi) / (2 chi);
//   mb = (e_th - i e_ph) / sqrt(2), Gram-Schmidt in gamma on x^i,
//   (-y, x, 0) and (x z, y z, -(x^2 + y^2)), in that order.
// dv: the derivative provider (stencils of the state, or the y/z pre-pass
// arrays as in the RHS).  x: the cell centre; 0 on the z axis, where the
// tetrad is undefined.
template <int ORD, class SRC, class DV>
__device__ __forceinline__ void psi4_point(const SRC &s, const DV &dv, double ichi, const double x[3],
                                           double out[2]) {
  using R = double;
  out[0] = out[1] = 0.0;
  if (x[0] * x[0] + x[1] * x[1] == 0.0) return;
  const R K = s.val(KHAT) + 2.0 * s.val(THETA);
  R g[6], A[6], gi[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    g[q] = s.val(GXX + q);
    A[q] = s.val(AXX + q);
  }
  inverse_metric(g, gi);
  R dchi[3], dK[3], dGam[3][3], dg[3][6], dA[3][6];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    dchi[d] = dv.d1(CHI, d);
    dK[d] = dv.d1(KHAT, d) + 2.0 * dv.d1(THETA, d);
#pragma unroll
    for (int i = 0; i < 3; ++i) dGam[d][i] = dv.d1(GAMX + i, d);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      dg[d][q] = dv.d1(GXX + q, d);
      dA[d][q] = dv.d1(AXX + q, d);
    }
  }
  R Gl[3][6], Gu[3][6], Gd[3];
  christoffel(gi, dg, Gl, Gu, Gd);
  R DDchi[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int q = S6(i, j);
      R ddc = i == j ? dv.d2(CHI, i) : dv.mix(CHI, i, j);
      DDchi[q] = ddc - (Gu[0][q] * dchi[0] + Gu[1][q] * dchi[1] + Gu[2][q] * dchi[2]);
    }
  R Ric[6];
  ricci(dv, ichi, g, gi, dchi, dg, dGam, Gl, Gu, Gd, DDchi, Ric);

  // physical metric and extrinsic curvature
  R gam[6], gamu[6], Kd[6], dKd[3][6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    gam[q] = g[q] * ichi;
    gamu[q] = gi[q] / ichi;
    Kd[q] = fma(g[q], K * (1.0 / 3.0), A[q]) * ichi;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int q = 0; q < 6; ++q)
      dKd[d][q] = (dA[d][q] + (dg[d][q] * K + g[q] * dK[d]) * (1.0 / 3.0) - Kd[q] * dchi[d]) * ichi;
  // Christoffels of gamma
  R gd[3], Gp[3][6];
#pragma unroll
  for (int m = 0; m < 3; ++m) gd[m] = gi[S6(m, 0)] * dchi[0] + gi[S6(m, 1)] * dchi[1] + gi[S6(m, 2)] * dchi[2];
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int l = k; l < 3; ++l) {
        const int q = S6(k, l);
        const R c = (m == k ? dchi[l] : 0.0) + (m == l ? dchi[k] : 0.0) - g[q] * gd[m];
        Gp[m][q] = Gu[m][q] - 0.5 * ichi * c;
      }
  // E_ij
  R E[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      R kk = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) kk += Kd[S6(i, k)] * gamu[S6(k, l)] * Kd[S6(l, j)];
      E[S6(i, j)] = Ric[S6(i, j)] + K * Kd[S6(i, j)] - kk;
    }
  // D_k K_lj and its curl C^m_j
  R DK[3][3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        R v = dKd[k][S6(l, j)];
#pragma unroll
        for (int m = 0; m < 3; ++m) v -= Gp[m][S6(k, l)] * Kd[S6(m, j)] + Gp[m][S6(k, j)] * Kd[S6(l, m)];
        DK[k][l][j] = v;
      }
  const R detg = g[0] * (g[3] * g[5] - g[4] * g[4]) - g[1] * (g[1] * g[5] - g[4] * g[2]) +
                 g[2] * (g[1] * g[4] - g[3] * g[2]);
  const R isq = 1.0 / (sqrt(detg) * ichi * sqrt(ichi));  // 1 / sqrt(det gamma)
  R C[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    C[0][j] = (DK[1][2][j] - DK[2][1][j]) * isq;
    C[1][j] = (DK[2][0][j] - DK[0][2][j]) * isq;
    C[2][j] = (DK[0][1][j] - DK[1][0][j]) * isq;
  }
  R Bt[3][3], B[6];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Bt[i][j] = gam[S6(i, 0)] * C[0][j] + gam[S6(i, 1)] * C[1][j] + gam[S6(i, 2)] * C[2][j];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) B[S6(i, j)] = 0.5 * (Bt[i][j] + Bt[j][i]);
  // tetrad: e[0] radial, e[1] phi, e[2] theta
  R e[3][3];
  const R u[3][3] = {{x[0], x[1], x[2]},
                     {-x[1], x[0], 0.0},
                     {x[0] * x[2], x[1] * x[2], -(x[0] * x[0] + x[1] * x[1])}};
  auto dotg = [&](const R *a, const R *b) {
    R v = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) v += gam[S6(i, j)] * a[i] * b[j];
    return v;
  };
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    R v[3] = {u[a][0], u[a][1], u[a][2]};
#pragma unroll
    for (int b = 0; b < a; ++b) {
      const R d = dotg(e[b], v);
#pragma unroll
      for (int i = 0; i < 3; ++i) v[i] -= d * e[b][i];
    }
    const R inv = 1.0 / sqrt(dotg(v, v));
#pragma unroll
    for (int i = 0; i < 3; ++i) e[a][i] = v[i] * inv;
  }
  auto quadf = [&](const R *X, const R *a, const R *b) {
    R v = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) v += X[S6(i, j)] * a[i] * b[j];
    return v;
  };
  const R *ph = e[1], *th = e[2];
  // mb^i mb^j = (th th - ph ph - i (th ph + ph th)) / 2
  out[0] = 0.5 * (quadf(E, th, th) - quadf(E, ph, ph)) - quadf(B, th, ph);
  out[1] = -quadf(E, th, ph) - 0.5 * (quadf(B, th, th) - quadf(B, ph, ph));
}

// ---- FP64 stage epilogue: RK update and algebraic constraint enforcement ----

// Float <-> double conversions on the integer pipe.  On this part FP64-pipe
// throughput is ~1/60 of FP32 and conversions otherwise issue to the FP64
// pipe.  float -> double is exact; double -> float rounds to nearest even.
// Both are branch-free and never fall back to a hardware conversion:
// subnormal results/operands are flushed to a signed zero, infinities and
// NaN are preserved (a NaN keeps the quiet bit).
__device__ __forceinline__ double f2d_int(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t e = (b >> 23) & 0xffu;
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  const uint64_t de = e == 0xffu ? 0x7ffull : (uint64_t)(e + 896u);
  const uint64_t d = sign | (de << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)(e == 0u ? sign : d));
}

__device__ __forceinline__ float d2f_int(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const int ef = e - 896;  // biased float exponent
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 mantissa bits
  const uint32_t rest = lo & 0x1fffffffu;                    // 29 dropped bits
  uint32_t f = sign | ((uint32_t)ef << 23) | m;
  f += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;  // carry may reach inf
  const uint32_t inf_nan = sign | 0x7f800000u | ((b & 0xfffffffffffffull) ? 0x400000u : 0u);
  f = e == 0x7ff ? inf_nan : (ef >= 255 ? (sign | 0x7f800000u) : (ef <= 0 ? sign : f));
  return __uint_as_float(f);
}

// x^(-1/3) for x > 0: FP32 seed, then Newton steps y <- y (4 - x y^3) / 3 in
// FP64 (each step squares the relative error: 2^-23 -> 2^-45 -> rounding).
template <int NEWTON>
__device__ __forceinline__ double rcbrt_newton(double x) {
  double y = f2d_int(rcbrtf(d2f_int(x)));
#pragma unroll
  for (int it = 0; it < NEWTON; ++it) {
    const double y3 = y * y * y;
    y = y * fma(-x, y3, 4.0) * (1.0 / 3.0);
  }
  return y;
}

// gt <- s gt with s = det(gt)^(-1/3); At <- At - gt tr(At)/3, the trace over
// the new inverse metric adj(s gt)/det(s gt) = s^2 adj(gt) (no division).
template <int NEWTON>
__device__ __forceinline__ void enforce(double v[NF]) {
  const double g0 = v[GXX], g1 = v[GXY], g2 = v[GXZ], g3 = v[GYY], g4 = v[GYZ], g5 = v[GZZ];
  const double a0 = g3 * g5 - g4 * g4, a1 = g2 * g4 - g1 * g5, a2 = g1 * g4 - g2 * g3;
  const double a3 = g0 * g5 - g2 * g2, a4 = g1 * g2 - g0 * g4, a5 = g0 * g3 - g1 * g1;
  const double det = g0 * a0 + g1 * a1 + g2 * a2;
  const double s = rcbrt_newton<NEWTON>(det);
  const double tr = s * s * (a0 * v[AXX] + a3 * v[AYY] + a5 * v[AZZ] +
                             2.0 * (a1 * v[AXY] + a2 * v[AXZ] + a4 * v[AYZ]));
  const double t3 = s * tr * (1.0 / 3.0);  // (s gt_ij) tr / 3 = gt_ij t3
  v[AXX] -= g0 * t3; v[AXY] -= g1 * t3; v[AXZ] -= g2 * t3;
  v[AYY] -= g3 * t3; v[AYZ] -= g4 * t3; v[AZZ] -= g5 * t3;
  v[GXX] = g0 * s; v[GXY] = g1 * s; v[GXZ] = g2 * s;
  v[GYY] = g3 * s; v[GYZ] = g4 * s; v[GZZ] = g5 * s;
}

// Field f of a register at one cell (u0 or the accumulator), read where it
// is used.
struct GlobalField {
  const double *p;
  int64_t off;
  int32_t S;
  __device__ __forceinline__ double operator()(int f) const { return p[off + (int64_t)f * S]; }
};

// RK4 stage update of one cell and enforcement, then the stores.  FP64 mode:
// FP64 fused multiply-adds of the FP64 RHS.  FP32 mode: the increment c k of
// the FP32 RHS is formed in FP32 and added to the FP64 state / accumulator
// in FP64; the next stage also goes to the FP32 shadow (the shadow_shifted
// fields minus 1).
// u0f / accf give field f of u0 and of the accumulator: GlobalField (read
// where used), ArrayField (loaded beforehand, below) or a staged copy.
template <class R, class U0F, class ACCF>
__device__ __forceinline__ void stage_epilogue_from(const StageArgs &a, int32_t block, int64_t off, int32_t S,
                                                    const R k[NF], const U0F &u0f, const ACCF &accf) {
  constexpr bool F32 = sizeof(R) == 4;
  const double dt = a.mode == MODE_RHS ? 0.0 : a.dts[block];
  const double ca = a.fa * dt, cb = a.fb * dt;
  const float caf = (float)ca, cbf = (float)cb;
  if (a.mode == MODE_RHS) {
#pragma unroll
    for (int f = 0; f < NF; ++f) a.rhs_out[off + (int64_t)f * S] = F32 ? f2d_int(float(k[f])) : double(k[f]);
    return;
  }
  double v[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int64_t o = off + (int64_t)f * S;
    if constexpr (F32) {
      const double dn = f2d_int(caf * float(k[f]));
      const double da = f2d_int(cbf * float(k[f]));
      if (a.mode == MODE_S1) {
        const double u = u0f(f);
        a.acc[o] = u + da;
        v[f] = u + dn;
      } else if (a.mode == MODE_S23) {
        a.acc[o] = accf(f) + da;
        v[f] = u0f(f) + dn;
      } else {
        v[f] = accf(f) + da;
      }
    } else {
      const double kd = double(k[f]);
      if (a.mode == MODE_S1) {
        const double u = u0f(f);
        a.acc[o] = fma(cb, kd, u);
        v[f] = fma(ca, kd, u);
      } else if (a.mode == MODE_S23) {
        a.acc[o] = fma(cb, kd, accf(f));
        v[f] = fma(ca, kd, u0f(f));
      } else {
        v[f] = fma(cb, kd, accf(f));
      }
    }
  }
  enforce<F32 ? 1 : 2>(v);
  if (a.next32 == nullptr) {
#pragma unroll
    for (int f = 0; f < NF; ++f) a.next[off + (int64_t)f * S] = v[f];
  } else {
    if (a.next_full) {
#pragma unroll
      for (int f = 0; f < NF; ++f) a.next[off + (int64_t)f * S] = v[f];
    } else {
      a.next[off] = v[CHI];
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const double w = shadow_shifted(f) ? v[f] - 1.0 : v[f];
      a.next32[off + (int64_t)f * S] = d2f_int(w);
    }
  }
}

template <class R>
__device__ __forceinline__ void stage_epilogue(const StageArgs &a, int32_t block, int64_t off, int32_t S,
                                               const R k[NF]) {
  stage_epilogue_from<R>(a, block, off, S, k, GlobalField{a.u0, off, S}, GlobalField{a.acc, off, S});
}

// The stage update with every u0 / accumulator value the stage reads loaded
// first, all at once (44 independent FP64 loads in flight per thread instead
// of a few at a time): for kernels with the registers to hold them.
struct ArrayField {
  const double *v;
  __device__ __forceinline__ double operator()(int f) const { return v[f]; }
};
struct StageOperands {
  double u0[NF], acc[NF];
  __device__ __forceinline__ void load(const StageArgs &a, int64_t off, int32_t S) {
    const bool need_u0 = a.mode == MODE_S1 || a.mode == MODE_S23;
    const bool need_acc = a.mode == MODE_S23 || a.mode == MODE_S4;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      u0[f] = need_u0 ? a.u0[off + (int64_t)f * S] : 0.0;
      acc[f] = need_acc ? a.acc[off + (int64_t)f * S] : 0.0;
    }
  }
};
template <class R>
__device__ __forceinline__ void stage_epilogue_preloaded(const StageArgs &a, int32_t block, int64_t off, int32_t S,
                                                         const R k[NF], const StageOperands &op) {
  stage_epilogue_from<R>(a, block, off, S, k, ArrayField{op.u0}, ArrayField{op.acc});
}

// 1/max(chi, floor) in FP64 for the FP32 algebra: integer compare (both
// operands positive or chi negative, so the bit patterns order like the
// values), FP32 reciprocal seed, one FP64 Newton step, rounded to FP32.
__device__ __forceinline__ float inv_chi_f32(double chi, double floor_) {
  const double c = __double_as_longlong(chi) > __double_as_longlong(floor_) ? chi : floor_;
  const double r0 = f2d_int(__frcp_rn(d2f_int(c)));
  const double e = fma(-c, r0, 1.0);
  return d2f_int(fma(r0, e, r0));
}

}  // namespace z4c
