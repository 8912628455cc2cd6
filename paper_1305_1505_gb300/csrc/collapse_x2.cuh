// Two particles at once: the FP32 per-particle arithmetic of collapse.cuh
// (eigenvalues, then the collapse time F = 1 / D(t_coll) of Sec. 2.1.1, Eq. F)
// on a pair of particles held in the two lanes of float2 values, with the
// packed single-precision instructions of sm_100-class GPUs
// (add/sub/mul/fma.rn.f32x2: one issued instruction for two lanes).  The z
// pass is bound by instruction issue, and the two particles a thread holds
// run the same branch-free formulas, so packing them halves the issued
// floating-point arithmetic.  Square roots, reciprocals, sine/cosine and
// exp2/log2 have no packed form and run per lane, as do compares and selects.
//
// The formulas and their order are those of eig3<float>, largest_root_iter,
// no_root_from and collapse_main in collapse.cuh (see there for the model and
// the reading of the paper); only the rounding of a few contracted products
// differs, so results agree with the scalar code to FP32 rounding, not bit
// for bit.  The rare minor-axis solve (collapse_rare) and the FP64 redo stay
// scalar.
#pragma once
#include <cuda_runtime.h>

#include "collapse.cuh"
#include "packed.cuh"

namespace pin {
namespace x2 {

// per-lane helpers
__device__ __forceinline__ float2 sqrt_approx(float2 a) {
  return make_float2(M<float>::sqrt_approx(a.x), M<float>::sqrt_approx(a.y));
}
__device__ __forceinline__ float2 cbrt_approx(float2 a) {
  return make_float2(M<float>::cbrt_approx(a.x), M<float>::cbrt_approx(a.y));
}
__device__ __forceinline__ float2 div(float2 a, float2 b) {
  return make_float2(M<float>::div_(a.x, b.x), M<float>::div_(a.y, b.y));
}
__device__ __forceinline__ float2 abs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }

}  // namespace x2

// eig3<float> of two symmetric matrices h[c] = (particle 0, particle 1),
// c = xx, yy, zz, xy, xz, yz; lam sorted per lane, largest first.  Returns the
// per-lane |r| (near 1: a near-degenerate pair, see eig3).
__device__ __forceinline__ float2 eig3_x2(const float2 h[6], float2 lam[3]) {
  using namespace x2;
  const float2 q = mul(add(add(h[0], h[1]), h[2]), splat(1.0f / 3.0f));
  const float2 b0 = sub(h[0], q), b1 = sub(h[1], q), b2 = sub(h[2], q);
  const float2 off = fma(h[5], h[5], fma(h[4], h[4], mul(h[3], h[3])));
  const float2 p2 = fma(splat(2.0f), off, fma(b2, b2, fma(b1, b1, mul(b0, b0))));
  const bool iso0 = !(p2.x > 0.0f), iso1 = !(p2.y > 0.0f);
  const float2 p6 = mul(p2, splat(1.0f / 6.0f));
  const float2 p = make_float2(M<float>::sqrt_(iso0 ? 0.0f : p6.x), M<float>::sqrt_(iso1 ? 0.0f : p6.y));
  // det(A - qI)
  const float2 t1 = sub(mul(b1, b2), mul(h[5], h[5]));
  const float2 t2 = sub(mul(h[3], b2), mul(h[5], h[4]));
  const float2 t3 = sub(mul(h[3], h[5]), mul(b1, h[4]));
  const float2 det = sub(fma(h[4], t3, mul(b0, t1)), mul(h[3], t2));
  const float2 den = mul(mul(splat(2.0f), p), mul(p, p));
  float2 r = div(det, den);
  r.x = iso0 ? 1.0f : fminf(fmaxf(r.x, -1.0f), 1.0f);
  r.y = iso1 ? 1.0f : fminf(fmaxf(r.y, -1.0f), 1.0f);
  // acos (Abramowitz & Stegun 4.4.46, as M<float>::acos_), lanes in parallel
  const float2 ax = abs(r);
  float2 poly = splat(-0.0012624911f);
  poly = fma(poly, ax, splat(0.0066700901f));
  poly = fma(poly, ax, splat(-0.0170881256f));
  poly = fma(poly, ax, splat(0.0308918810f));
  poly = fma(poly, ax, splat(-0.0501743046f));
  poly = fma(poly, ax, splat(0.0889789874f));
  poly = fma(poly, ax, splat(-0.2145988016f));
  poly = fma(poly, ax, splat(1.5707963050f));
  const float2 om = sub(splat(1.0f), ax);
  const float2 ac = mul(make_float2(M<float>::sqrt_(fmaxf(om.x, 0.0f)), M<float>::sqrt_(fmaxf(om.y, 0.0f))), poly);
  const float2 acs = make_float2(r.x < 0.0f ? 3.14159265358979f - ac.x : ac.x,
                                 r.y < 0.0f ? 3.14159265358979f - ac.y : ac.y);
  const float2 phi = mul(acs, splat(1.0f / 3.0f));
  float2 sn, cs;
  M<float>::sincos_(phi.x, &sn.x, &cs.x);
  M<float>::sincos_(phi.y, &sn.y, &cs.y);
  // cos(phi + 2 pi/3) = -cos(phi)/2 - (sqrt(3)/2) sin(phi)
  const float2 l0 = fma(mul(splat(2.0f), p), cs, q);
  const float2 l2 = sub(q, mul(p, fma(splat(1.7320508075688772935f), sn, cs)));
  lam[0] = l0;
  lam[2] = l2;
  lam[1] = sub(sub(mul(splat(3.0f), q), l0), l2);
  return abs(r);
}

// largest_root_iter<float> for two cubics g(F) = F^3 - c1 F^2 - c2 F - c3.
__device__ __forceinline__ float2 largest_root_iter_x2(float2 c1, float2 c2, float2 c3, float2& kappa) {
  using namespace x2;
  const float2 s = mul(c1, splat(1.0f / 3.0f));
  const float2 np = fma(c1, s, c2);                                   // -p
  const float2 nq = fma(mul(splat(2.0f), s), mul(s, s), fma(c2, s, c3));  // -q
  const float2 hq = mul(nq, splat(-0.5f));
  const float2 tp = mul(np, splat(-1.0f / 3.0f));
  const float2 disc = fma(hq, hq, mul(mul(tp, tp), tp));
  const bool right0 = disc.x <= 0.0f || nq.x >= 0.0f, right1 = disc.y <= 0.0f || nq.y >= 0.0f;
  const float2 up = add(add(s, sqrt_approx(np)), cbrt_approx(nq));
  const bool none0 = !right0 && c3.x <= 0.0f, none1 = !right1 && c3.y <= 0.0f;
  float2 x = make_float2(right0 ? up.x : 0.0f, right1 ? up.y : 0.0f);
  const float2 nc1 = mul(c1, splat(-1.0f)), nc2 = mul(c2, splat(-1.0f)), nc3 = mul(c3, splat(-1.0f));
  const float2 m2c1 = mul(c1, splat(-2.0f));
  float2 step = splat(0.0f);
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const float2 g = fma(fma(add(x, nc1), x, nc2), x, nc3);
    const float2 dg = fma(fma(splat(3.0f), x, m2c1), x, nc2);
    const float2 nd2h = fma(splat(-3.0f), x, c1);                     // -g''/2
    const float2 den = fma(dg, dg, mul(g, nd2h));
    const float2 num = mul(g, dg);
    step = div(num, make_float2(den.x > 1e-30f ? den.x : 1e-30f, den.y > 1e-30f ? den.y : 1e-30f));
    x = sub(x, step);
  }
  // conditioning |g'(x)| / (3x^2 + 2|c1||x| + |c2|) (root_kappa)
  const float2 dg = fma(fma(splat(3.0f), x, m2c1), x, nc2);
  const float2 ax = abs(x);
  const float2 scale = fma(mul(splat(2.0f), abs(c1)), ax, fma(mul(splat(3.0f), x), x, abs(c2)));
  const float2 kap = div(abs(dg), make_float2(scale.x > 0.0f ? scale.x : 1.0f, scale.y > 0.0f ? scale.y : 1.0f));
  const float2 as = abs(step);
  const float2 lim = fma(splat(2e-6f), ax, splat(1e-12f));
  kappa.x = none0 ? 1.0f : (as.x > lim.x ? 0.0f : (scale.x > 0.0f ? kap.x : 1.0f));
  kappa.y = none1 ? 1.0f : (as.y > lim.y ? 0.0f : (scale.y > 0.0f ? kap.y : 1.0f));
  return make_float2((none0 || !(x.x > 0.0f)) ? 0.0f : x.x, (none1 || !(x.y > 0.0f)) ? 0.0f : x.y);
}

// no_root_from<float> for two cubics and two thresholds t; bit 0 / bit 1 of
// the result: lane 0 / lane 1 has no real root at or above its t.
__device__ __forceinline__ unsigned no_root_from_x2(float2 c1, float2 c2, float2 c3, float2 t) {
  using namespace x2;
  const float2 gt = sub(mul(sub(mul(sub(t, c1), t), c2), t), c3);
  const float2 d = fma(c1, c1, mul(splat(3.0f), c2));
  const float2 fs = mul(add(c1, sqrt_approx(d)), splat(1.0f / 3.0f));
  const float2 gs = sub(mul(sub(mul(sub(fs, c1), fs), c2), fs), c3);
  const bool n0 = (gt.x > 0.0f) & ((d.x < 0.0f) | (fs.x <= t.x) | (gs.x > 0.0f));
  const bool n1 = (gt.y > 0.0f) & ((d.y < 0.0f) | (fs.y <= t.y) | (gs.y > 0.0f));
  return (n0 ? 1u : 0u) | (n1 ? 2u : 0u);
}

// Per-pair state between the common part and the rare minor-axis solve.
struct CollapseStateX2 {
  float2 best, kappa, corr;
  float2 c[2][3];  // coefficients of the two smaller-eigenvalue axes
  unsigned need;   // bit (2 a + lane): axis a + 1 of that lane may collapse first
};

// First part of collapse_main<float> for two particles: the coefficients of
// the three axes (c0 for the axis of the largest eigenvalue, st.c for the
// others) and the quasi-spherical correction term st.corr.
__device__ __forceinline__ void collapse_prep_x2(const float2 lam[3], const CollapseConsts<float>& cc,
                                                 CollapseStateX2& st, float2 c0[3]) {
  using namespace x2;
  const float2 mu1 = add(add(lam[0], lam[1]), lam[2]);
  const float2 mu3 = mul(mul(lam[0], lam[1]), lam[2]);
  const float2 s12 = add(lam[1], lam[2]), s02 = add(lam[0], lam[2]), s01 = add(lam[0], lam[1]);
  const float2 half = splat(0.5f);
  const float2 e0 = mul(mul(half, lam[0]), s12);
  const float2 e1 = mul(mul(half, lam[1]), s02);
  const float2 e2 = mul(mul(half, lam[2]), s01);
  const float2 k37 = splat(3.0f / 7.0f), k1084 = splat(10.0f / 84.0f);
  const float2 nmu3 = mul(mu3, splat(-1.0f / 9.0f));
  // axis i: c1 = lam_i, c2 = (3/7) e_i, c3 = (10/84)(lam_i (e_j + e_k) + e_i (lam_j + lam_k)) - mu3/9
  c0[0] = lam[0];
  c0[1] = mul(k37, e0);
  c0[2] = fma(k1084, fma(e0, s12, mul(lam[0], add(e1, e2))), nmu3);
  st.c[0][0] = lam[1];
  st.c[0][1] = mul(k37, e1);
  st.c[0][2] = fma(k1084, fma(e1, s02, mul(lam[1], add(e2, e0))), nmu3);
  st.c[1][0] = lam[2];
  st.c[1][1] = mul(k37, e2);
  st.c[1][2] = fma(k1084, fma(e2, s01, mul(lam[2], add(e0, e1))), nmu3);
  // quasi-spherical correction: z = eps / 0.1
  const float2 num = mul(splat(10.0f), sub(lam[0], lam[2]));
  const float2 z = div(num, make_float2(mu1.x > 0.0f ? mu1.x : 1.0f, mu1.y > 0.0f ? mu1.y : 1.0f));
  const float2 nz2 = mul(mul(z, z), splat(-1.0f));
  const float2 w = make_float2(M<float>::exp_(nz2.x), M<float>::exp_(nz2.y));
  const float2 cw = mul(mul(mu1, splat(cc.dcorr)), w);
  st.corr.x = (cc.correction && mu1.x > 0.0f) ? cw.x : 0.0f;
  st.corr.y = (cc.correction && mu1.y > 0.0f) ? cw.y : 0.0f;
}

// Second part: the largest root of the axis-0 cubic (st.best, st.kappa) and
// the exact test whether the two other axes may collapse first (st.need).
__device__ __forceinline__ void collapse_root_x2(const float2 c0[3], CollapseStateX2& st) {
  st.best = largest_root_iter_x2(c0[0], c0[1], c0[2], st.kappa);
  const unsigned n0 = no_root_from_x2(st.c[0][0], st.c[0][1], st.c[0][2], st.best);
  const unsigned n1 = no_root_from_x2(st.c[1][0], st.c[1][1], st.c[1][2], st.best);
  st.need = (~n0 & 3u) | ((~n1 & 3u) << 2);
}

// collapse_main<float> for two particles.
__device__ __forceinline__ void collapse_main_x2(const float2 lam[3], const CollapseConsts<float>& cc,
                                                 CollapseStateX2& st) {
  float2 c0[3];
  collapse_prep_x2(lam, cc, st, c0);
  collapse_root_x2(c0, st);
}

// Which lanes cannot reach F > fm (bit 0 / bit 1): F = max_i F_i + corr with
// F_i >= 0 the largest root of axis i (clamped at 0), so F < fm when
// t = fm - corr >= 0 and no axis cubic has a real root at or above t.  The
// test runs at t (1 - 1e-5), below t by more than the FP32 error of a root, so
// that a lane it clears could not have been updated by the full computation
// (nor by its FP64 redo).  Exact up to rounding, like no_root_from.
__device__ __forceinline__ unsigned cannot_beat_x2(const float2 c0[3], const CollapseStateX2& st, float2 fm) {
  using namespace x2;
  const float2 t = mul(sub(fm, st.corr), splat(1.0f - 1e-5f));
  const unsigned a0 = no_root_from_x2(c0[0], c0[1], c0[2], t);
  const unsigned a1 = no_root_from_x2(st.c[0][0], st.c[0][1], st.c[0][2], t);
  const unsigned a2 = no_root_from_x2(st.c[1][0], st.c[1][1], st.c[1][2], t);
  const unsigned nonneg = (t.x >= 0.0f ? 1u : 0u) | (t.y >= 0.0f ? 2u : 0u);
  return a0 & a1 & a2 & nonneg;
}

// One lane of a pair state as the scalar state of collapse.cuh (for the rare
// minor-axis solve).
__device__ __forceinline__ CollapseState<float> lane_state(const CollapseStateX2& s, int lane) {
  CollapseState<float> o;
  o.best = lane ? s.best.y : s.best.x;
  o.kappa = lane ? s.kappa.y : s.kappa.x;
  o.corr = lane ? s.corr.y : s.corr.x;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
#pragma unroll
    for (int k = 0; k < 3; ++k) o.c[a][k] = lane ? s.c[a][k].y : s.c[a][k].x;
    o.need[a] = (s.need >> (2 * a + lane)) & 1u;
  }
  return o;
}

// collapse_from_eigs<float> of two particles: F per lane and the conditioning
// of the root that set it.
__device__ __forceinline__ float2 collapse_from_eigs_x2(const float2 lam[3], const CollapseConsts<float>& cc,
                                                        float2& kappa) {
  CollapseStateX2 st;
  collapse_main_x2(lam, cc, st);
  float2 F;
#pragma unroll
  for (int lane = 0; lane < 2; ++lane) {
    CollapseState<float> s = lane_state(st, lane);
    if (s.need[0] || s.need[1]) collapse_rare<float>(s);
    (lane ? F.y : F.x) = s.best + s.corr;
    (lane ? kappa.y : kappa.x) = s.kappa;
  }
  return F;
}

}  // namespace pin
