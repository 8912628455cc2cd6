// Per-particle eigenvalues of the deformation tensor and the ellipsoidal
// collapse time F = 1 / D(t_coll) (Sec. 2.1.1, Eq. F), templated on the
// arithmetic type so that the same code runs in FP32 and, for the rare
// ill-conditioned particles, in FP64.
//
// Collapse model (ellipsoidal truncation of third-order LPT with the growing
// mode D as the clock; the paper cites the formulas to earlier work, this is
// the reading used throughout): in the eigenframe, with mu1 = sum lambda,
// mu2 = sum_{i<j} lambda_i lambda_j, mu3 = prod lambda and
// e_i = lambda_i (lambda_j + lambda_k) / 2, axis i is compressed by
//   a_i(D) = c1 D + c2 D^2 + c3 D^3,
//   c1 = lambda_i, c2 = (3/7) e_i,
//   c3 = (10/84)(lambda_i (e_j + e_k) + e_i (lambda_j + lambda_k)) - mu3 / 9,
// and orbit crossing of the first axis is the smallest D > 0 with a_i(D) = 1
// over the three axes.  Dividing a_i(D) = 1 by D^3 turns it into the monic
// cubic in F = 1/D
//   g_i(F) = F^3 - c1 F^2 - c2 F - c3 = 0,
// so the smallest positive D is the LARGEST positive real root F of g_i, and
// F = max_i F_i (0 when no axis collapses).  That root is taken in closed form
// (Cardano / trigonometric) and polished by Newton steps on g_i.
//
// Quasi-spherical correction (Sec. 2.1.1): for mu1 > 0,
//   F += mu1 (1/delta_c - 1/x3) exp(-(eps/0.1)^2),  eps = (lambda1 - lambda3)/|mu1|,
// which makes a sphere collapse exactly at F = delta/delta_c; x3 is the
// uncorrected spherical root (x/3 + x^2/21 + 23 x^3/1701 = 1).
#pragma once
#include <cuda_runtime.h>
#include <cmath>

namespace pin {

// Arithmetic of one precision.  FP64 (the redo of ill-conditioned particles)
// uses the accurate library functions.  FP32 keeps the hot loop short:
//  - acos: Abramowitz & Stegun 4.4.46 (Hastings) sqrt(1-x) * (degree-7
//    polynomial), |error| <= 2e-8 on [0, 1], mirrored for x < 0;
//  - sin/cos of arguments in [0, pi] and exp of non-positive arguments: the
//    hardware approximations (absolute error ~2^-21 for sin/cos);
//  - cbrt: exp2(log2|x| / 3) from the hardware approximations, then one
//    Newton step u <- (2u + x/u^2)/3, which squares the relative error;
//  - division: the two-ulp fast form.
// On the host (unit tests) the same formulas run with the C++ library
// standing in for the hardware approximations.
#ifdef __CUDA_ARCH__
// single-instruction approximations (PTX sqrt/lg2/ex2 .approx): relative error
// a few ulp; sqrt(0) = 0, lg2(0) = -inf, ex2(-inf) = 0
__device__ __forceinline__ float ptx_sqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ptx_lg2(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ptx_ex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
#endif

template <typename T> struct M;
template <> struct M<float> {
  // approximate square root of x >= 0 (a few ulp, no special-case branches)
  __host__ __device__ __forceinline__ static float sqrt_(float x) {
#ifdef __CUDA_ARCH__
    return ptx_sqrt(x);
#else
    return std::sqrt(x);
#endif
  }
  __host__ __device__ __forceinline__ static float div_(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
  }
  __host__ __device__ __forceinline__ static float acos_(float x) {
    const float ax = fabsf(x);
    float poly = -0.0012624911f;
    poly = fmaf(poly, ax, 0.0066700901f);
    poly = fmaf(poly, ax, -0.0170881256f);
    poly = fmaf(poly, ax, 0.0308918810f);
    poly = fmaf(poly, ax, -0.0501743046f);
    poly = fmaf(poly, ax, 0.0889789874f);
    poly = fmaf(poly, ax, -0.2145988016f);
    poly = fmaf(poly, ax, 1.5707963050f);
    const float r = sqrt_(fmaxf(1.0f - ax, 0.0f)) * poly;
    return x < 0.0f ? 3.14159265358979f - r : r;
  }
  __host__ __device__ __forceinline__ static void sincos_(float x, float* sn, float* cs) {
#ifdef __CUDA_ARCH__
    __sincosf(x, sn, cs);
#else
    *sn = std::sin(x);
    *cs = std::cos(x);
#endif
  }
  __host__ __device__ __forceinline__ static float cos_(float x) {
#ifdef __CUDA_ARCH__
    return __cosf(x);
#else
    return std::cos(x);
#endif
  }
  __host__ __device__ __forceinline__ static float exp_(float x) {
#ifdef __CUDA_ARCH__
    return __expf(x);
#else
    return std::exp(x);
#endif
  }
  // approximate sqrt / cbrt of max(x, 0) (relative error ~1e-7 / ~1e-6): bounds only
  __host__ __device__ __forceinline__ static float sqrt_approx(float x) {
#ifdef __CUDA_ARCH__
    return ptx_sqrt(fmaxf(x, 0.0f));
#else
    return x > 0.0f ? std::sqrt(x) : 0.0f;
#endif
  }
  __host__ __device__ __forceinline__ static float cbrt_approx(float x) {
#ifdef __CUDA_ARCH__
    return ptx_ex2(ptx_lg2(fmaxf(x, 0.0f)) * (1.0f / 3.0f));
#else
    return x > 0.0f ? std::cbrt(x) : 0.0f;
#endif
  }
  __host__ __device__ __forceinline__ static float cbrt_(float x) {
    if (x == 0.0f) return 0.0f;
    const float ax = fabsf(x);
#ifdef __CUDA_ARCH__
    float u = ptx_ex2(ptx_lg2(ax) * (1.0f / 3.0f));
#else
    float u = std::exp2(std::log2(ax) * (1.0f / 3.0f));
#endif
    u = (2.0f * u + div_(ax, u * u)) * (1.0f / 3.0f);
    return x < 0.0f ? -u : u;
  }
};
template <> struct M<double> {
  __host__ __device__ __forceinline__ static double sqrt_(double x) { return sqrt(x); }
  __host__ __device__ __forceinline__ static double div_(double a, double b) { return a / b; }
  __host__ __device__ __forceinline__ static double acos_(double x) { return acos(x); }
  __host__ __device__ __forceinline__ static void sincos_(double x, double* sn, double* cs) {
    *sn = sin(x);
    *cs = cos(x);
  }
  __host__ __device__ __forceinline__ static double cos_(double x) { return cos(x); }
  __host__ __device__ __forceinline__ static double exp_(double x) { return exp(x); }
  __host__ __device__ __forceinline__ static double cbrt_(double x) { return cbrt(x); }
  __host__ __device__ __forceinline__ static double sqrt_approx(double x) { return x > 0.0 ? sqrt(x) : 0.0; }
  __host__ __device__ __forceinline__ static double cbrt_approx(double x) { return x > 0.0 ? cbrt(x) : 0.0; }
};

// Closed-form eigenvalues of the symmetric 3x3 matrix
// h = (xx, yy, zz, xy, xz, yz), sorted lam[0] >= lam[1] >= lam[2]
// (trigonometric solution of the characteristic cubic, Smith 1961).
// Returns |r| = |det(B)|/2, B = (A - qI)/p; |r| -> 1 marks a near-degenerate
// pair, whose split the trigonometric form resolves poorly in FP32.
template <typename T>
__host__ __device__ __forceinline__ T eig3(const T h[6], T lam[3]) {
  using F = M<T>;
  const T third = T(1) / T(3);
  const T q = (h[0] + h[1] + h[2]) * third;
  const T b0 = h[0] - q, b1 = h[1] - q, b2 = h[2] - q;
  const T off = h[3] * h[3] + h[4] * h[4] + h[5] * h[5];
  const T p2 = b0 * b0 + b1 * b1 + b2 * b2 + T(2) * off;
  // p2 == 0 (a multiple of the identity) gives p = 0 and three equal values
  // through the same formulas, with r forced to 1 (flagged, redone in FP64)
  const bool iso = !(p2 > T(0));
  const T p = F::sqrt_(iso ? T(0) : p2 * (T(1) / T(6)));
  // det(A - qI)
  const T det = b0 * (b1 * b2 - h[5] * h[5]) - h[3] * (h[3] * b2 - h[5] * h[4]) +
                h[4] * (h[3] * h[5] - b1 * h[4]);
  T r = iso ? T(1) : F::div_(det, T(2) * p * p * p);
  r = r > T(1) ? T(1) : (r < T(-1) ? T(-1) : r);
  const T phi = F::acos_(r) * third;
  T sn, cs;
  F::sincos_(phi, &sn, &cs);
  // cos(phi + 2 pi/3) = -cos(phi)/2 - (sqrt(3)/2) sin(phi)
  const T l0 = q + T(2) * p * cs;
  const T l2 = q - p * (cs + T(1.7320508075688772935) * sn);
  lam[0] = l0;
  lam[2] = l2;
  lam[1] = T(3) * q - l0 - l2;
  return r < T(0) ? -r : r;
}

// Conditioning of a root x of g: |g'(x)| / (3x^2 + 2|c1|x + |c2|), small near
// a tangent crossing.
template <typename T>
__host__ __device__ __forceinline__ T root_kappa(T c1, T c2, T x) {
  using F = M<T>;
  const T dg = (T(3) * x - T(2) * c1) * x - c2;
  const T ac1 = c1 < T(0) ? -c1 : c1, ac2 = c2 < T(0) ? -c2 : c2, ax = x < T(0) ? -x : x;
  const T scale = T(3) * x * x + T(2) * ac1 * ax + ac2;
  return scale > T(0) ? F::div_(dg < T(0) ? -dg : dg, scale) : T(1);
}

// Largest real root of g(F) = F^3 - c1 F^2 - c2 F - c3, clamped at 0 from
// below (no positive root: the axis never collapses), without branches on the
// root structure: Halley's iteration from a point on the monotone side of the
// root.  With the depressed form t^3 + p t + q (F = t + c1/3):
//  - if there are three real roots, or q <= 0, the largest root lies right of
//    the inflection point c1/3, where g is convex and increasing; start at
//    U = c1/3 + sqrt(max(-p,0)) + cbrt(max(-q,0)), an upper bound (for
//    t >= a + b with a^2 >= -p, b^3 >= -q: t^3 + p t + q >= t(t^2 - a^2) - b^3
//    >= 2a^2 b + 3a b^2 >= 0);
//  - otherwise the single real root lies left of it, in the concave increasing
//    region; it is positive only if g(0) = -c3 < 0, and the iteration starts at 0.
// Four iterations reach ~1e-6 relative in FP32 on the coefficient ranges of
// smoothed Gaussian fields; near-tangent roots are flagged by kappa and redone.
template <typename T>
__host__ __device__ __forceinline__ T largest_root_iter(T c1, T c2, T c3, T& kappa) {
  using F = M<T>;
  const T third = T(1) / T(3);
  const T s = c1 * third;
  const T p = -c2 - c1 * s;
  const T q = -c3 - c2 * s - T(2) * s * s * s;
  const T hq = q * T(0.5), tp = p * third;
  const T disc = hq * hq + tp * tp * tp;
  const bool right = disc <= T(0) || q <= T(0);
  const T up = s + F::sqrt_approx(-p) + F::cbrt_approx(-q);
  const bool none = !right && c3 <= T(0);  // single root, and it is not positive
  T x = right ? up : T(0);
  T step = T(0);
  // Halley: x -= g g' / (g'^2 - g g''/2).  The denominator is floored at a
  // tiny positive value instead of tested: a degenerate step leaves a large
  // last step, which sends the particle to the FP64 redo below.
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const T g = ((x - c1) * x - c2) * x - c3;
    const T dg = (T(3) * x - T(2) * c1) * x - c2;
    const T d2h = T(3) * x - c1;
    const T den = dg * dg - g * d2h;
    step = F::div_(g * dg, den > T(1e-30) ? den : T(1e-30));
    x = x - step;
  }
  kappa = root_kappa<T>(c1, c2, x);
  // not converged after four steps: hand the particle to the FP64 redo
  const T ax = x < T(0) ? -x : x, as = step < T(0) ? -step : step;
  kappa = (as > T(2e-6) * ax + T(1e-12)) ? T(0) : kappa;
  kappa = none ? T(1) : kappa;
  return (none || !(x > T(0))) ? T(0) : x;
}

// Same root by the closed form (Cardano / trigonometric) with two Newton
// polishing steps; used in FP64, where the accurate library functions make it
// exact to rounding.
template <typename T>
__host__ __device__ __forceinline__ T largest_root_closed(T c1, T c2, T c3, T& kappa) {
  using F = M<T>;
  const T third = T(1) / T(3);
  const T s = c1 * third;
  const T p = -c2 - c1 * s;                                   // b - a^2/3
  const T q = -c3 - c2 * s - T(2) * s * s * s;                 // 2a^3/27 - ab/3 + c
  const T hq = q * T(0.5), tp = p * third;
  const T disc = hq * hq + tp * tp * tp;
  T t;
  if (disc <= T(0) && p < T(0)) {
    // three real roots t_k = m cos(theta/3 - 2 pi k/3); the largest is k = 0
    const T m = T(2) * F::sqrt_(-tp);
    T arg = F::div_(T(3) * q, p * m);
    arg = arg > T(1) ? T(1) : (arg < T(-1) ? T(-1) : arg);
    t = m * F::cos_(F::acos_(arg) * third);
  } else {
    // one real root: t = u - p/(3u), u the cube root of larger magnitude
    const T sd = F::sqrt_(disc > T(0) ? disc : T(0));
    const T w = hq >= T(0) ? -hq - sd : -hq + sd;
    const T u = F::cbrt_(w);
    t = (u != T(0)) ? u - F::div_(tp, u) : T(0);
  }
  T x = t + s;
  // Newton polish on g
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const T g = ((x - c1) * x - c2) * x - c3;
    const T dg = (T(3) * x - T(2) * c1) * x - c2;
    if (dg != T(0)) x = x - F::div_(g, dg);
  }
  kappa = root_kappa<T>(c1, c2, x);
  return x > T(0) ? x : T(0);
}

template <typename T>
__host__ __device__ __forceinline__ T largest_root(T c1, T c2, T c3, T& kappa) {
  if constexpr (sizeof(T) == 4) return largest_root_iter<T>(c1, c2, c3, kappa);
  else return largest_root_closed<T>(c1, c2, c3, kappa);
}

template <typename T>
struct CollapseConsts {
  T dcorr;   // 1/delta_c - 1/x3
  int correction;
};

// Upper bound on the collapse time F of a particle from two invariants of its
// deformation tensor h, without the eigenvalues.  With q = tr(h)/3 and
// 6 p^2 = tr((h - qI)^2), every eigenvalue lies in [q - 2p, q + 2p] (the
// deviations from q sum to zero and their squares to 6 p^2), so
// |lambda_i| <= L = |q| + 2p.  Then for every axis |c1| <= L,
// |c2| = (3/7)|e_i| <= (3/7) L^2 and |c3| <= (10/84)(2 L^3 + 2 L^3) + L^3/9
// < 0.5874 L^3, so g(F) >= F^3 - L F^2 - (3/7) L^2 F - 0.5874 L^3, which is
// increasing for F >= L and positive at F = 1.54 L (1.54^3 - 1.54^2 -
// (3/7) 1.54 - 0.5874 > 0.03): every axis root lies below 1.54 L.  The
// correction is at most max(mu1, 0) dcorr (mu1 = 3q, exp(-z^2) <= 1).
// Used to clear particles queued for the FP64 redo that cannot beat their
// running maximum.
constexpr double kRootBound = 1.54;
template <typename T>
__host__ __device__ __forceinline__ T collapse_bound(const T h[6], const CollapseConsts<T>& cc) {
  using F = M<T>;
  const T q = (h[0] + h[1] + h[2]) * (T(1) / T(3));
  const T b0 = h[0] - q, b1 = h[1] - q, b2 = h[2] - q;
  const T p2 = b0 * b0 + b1 * b1 + b2 * b2 + T(2) * (h[3] * h[3] + h[4] * h[4] + h[5] * h[5]);
  const T L = (q < T(0) ? -q : q) + T(2) * F::sqrt_approx(p2 * (T(1) / T(6)));
  const T mu1 = T(3) * q;
  const T corr = (cc.correction && mu1 > T(0) && cc.dcorr > T(0)) ? mu1 * cc.dcorr : T(0);
  return T(kRootBound) * L + corr;
}

// True when g(F) = F^3 - c1 F^2 - c2 F - c3 has no real root at or above T:
// g(T) > 0 and g stays positive beyond T, i.e. g' has no real root, or the
// right critical point F* = (c1 + sqrt(c1^2 + 3 c2))/3 lies at or below T, or
// g(F*) > 0 (g is increasing beyond F*).  Exact up to rounding, and far
// cheaper than solving the cubic.  Every term is evaluated (no early exits),
// so that the particles of a warp do not diverge on it.
template <typename T>
__host__ __device__ __forceinline__ bool no_root_from(T c1, T c2, T c3, T t) {
  using F = M<T>;
  const T gt = ((t - c1) * t - c2) * t - c3;
  const T d = c1 * c1 + T(3) * c2;
  const T fs = (c1 + F::sqrt_approx(d)) * (T(1) / T(3));
  const T gs = ((fs - c1) * fs - c2) * fs - c3;
  return (gt > T(0)) & ((d < T(0)) | (fs <= t) | (gs > T(0)));
}

// Coefficients (c1, c2, c3) of a_i(D) = c1 D + c2 D^2 + c3 D^3 for axis i.
template <typename T>
__host__ __device__ __forceinline__ void axis_coeffs(const T lam[3], const T e[3], T mu3, int i, T c[3]) {
  const int j = (i + 1) % 3, k = (i + 2) % 3;
  c[0] = lam[i];
  c[1] = T(3) / T(7) * e[i];
  c[2] = T(10) / T(84) * (lam[i] * (e[j] + e[k]) + e[i] * (lam[j] + lam[k])) - mu3 * (T(1) / T(9));
}

// Per-particle state between the two parts of the collapse computation.
template <typename T>
struct CollapseState {
  T best, kappa, corr;
  T c[2][3];     // coefficients of the two smaller-eigenvalue axes
  bool need[2];  // those axes may collapse first and must be solved
};

// Common part, free of branches on the data so that independent particles
// interleave: the axis of the largest eigenvalue, the exact test for the other
// two (no_root_from at its root), and the quasi-spherical correction term.
template <typename T>
__host__ __device__ __forceinline__ void collapse_main(const T lam[3], const CollapseConsts<T>& cc,
                                                       CollapseState<T>& st) {
  using F = M<T>;
  const T mu1 = lam[0] + lam[1] + lam[2];
  const T mu3 = lam[0] * lam[1] * lam[2];
  T e[3];
  e[0] = T(0.5) * lam[0] * (lam[1] + lam[2]);
  e[1] = T(0.5) * lam[1] * (lam[0] + lam[2]);
  e[2] = T(0.5) * lam[2] * (lam[0] + lam[1]);
  T c0[3];
  axis_coeffs<T>(lam, e, mu3, 0, c0);
  axis_coeffs<T>(lam, e, mu3, 1, st.c[0]);
  axis_coeffs<T>(lam, e, mu3, 2, st.c[1]);
  st.best = largest_root<T>(c0[0], c0[1], c0[2], st.kappa);
#pragma unroll
  for (int a = 0; a < 2; ++a) st.need[a] = !no_root_from<T>(st.c[a][0], st.c[a][1], st.c[a][2], st.best);
  const T z = F::div_(T(10) * (lam[0] - lam[2]), mu1 > T(0) ? mu1 : T(1));  // eps / 0.1
  const T w = F::exp_(-z * z);
  st.corr = (cc.correction && mu1 > T(0)) ? mu1 * cc.dcorr * w : T(0);
}

// Rare part: solve the smaller-eigenvalue axes that may collapse first.
template <typename T>
__host__ __device__ __forceinline__ void collapse_rare(CollapseState<T>& st) {
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    if (!st.need[a]) continue;
    T kap;
    const T Fi = largest_root<T>(st.c[a][0], st.c[a][1], st.c[a][2], kap);
    if (Fi > st.best) {
      st.best = Fi;
      st.kappa = kap;
    }
  }
}

// F for sorted eigenvalues lam; kappa_min receives the conditioning of the
// root that set F (1 when nothing collapses).  The axis of the largest
// eigenvalue is solved first; the other two are solved only when they can
// collapse earlier (no_root_from), which is rare.
template <typename T>
__host__ __device__ __forceinline__ T collapse_from_eigs(const T lam[3], const CollapseConsts<T>& cc,
                                                         T& kappa_min) {
  CollapseState<T> st;
  collapse_main<T>(lam, cc, st);
  if (st.need[0] || st.need[1]) collapse_rare<T>(st);
  kappa_min = st.kappa;
  return st.best + st.corr;
}

}  // namespace pin
