// kf_math.cuh -- per-track Kalman-filter arithmetic for one thread.
//
// The core operations of Kalman-filter tracking (Cerati et al., Sec. 2 and
// Sec. 2.1): propagate a track state and its symmetric 6x6 covariance to the
// next barrel layer, then compute the chi2 of a 3-D hit and apply the Kalman
// gain update.  Sec. 2.1 stresses symmetric storage, on-the-fly transposes
// and matrix elements known to be zero or one; here that is done at compile
// time: the covariance lives in registers as 21 packed values, and every
// product below touches only the structurally non-zero entries of the
// transport Jacobian (column z0 is e_z, row pz is e_pz).
//
// Multiply-adds are written as explicit fma_t, and the translation units
// that use this header are compiled without implicit contraction, so every
// kernel (per-layer, fused, plain-load or staged) rounds each track the same
// way and gives the same bits.  The same templates give T = float and
// T = double (the plain FP64 form).

// State (x, y, z, px, py, pz) in cm and GeV; a = q * 0.00299792458 * Bz.
// Helix:  theta = a s / p,
//   x(s)  = x0 + px0 sin(th)/a + py0 (1 - cos th)/a
//   y(s)  = y0 + py0 sin(th)/a - px0 (1 - cos th)/a,   z(s) = z0 + pz0 s / p
//   px(s) = px0 cos th + py0 sin th,   py(s) = py0 cos th - px0 sin th.
// sin(th)/a = (s/p) sinc(h) cos(h) and (1 - cos th)/a = (s/p) h sinc(h)^2
// with h = th/2: no 1/a and no 1 - cos cancellation.
// The path length s to radius R solves g(s) = x(s)^2 + y(s)^2 - R^2 = 0 by
// Newton iterations from a guess that keeps the curvature terms to second
// order (below).  The transport Jacobian is
// the surface one, J = dF/dx0|_s - (dF/ds)(dg/dx0|_s)/(dg/ds).
//
// Compiles for the host too, so that the same source can be exercised off
// the GPU.
#pragma once

#include <math.h>
#include <stdint.h>

#ifdef __CUDACC__
#define KF_HD __host__ __device__ __forceinline__
#else
#define KF_HD inline
#endif

namespace kf {

// per-track status bits (the ABI's KF_ST_* values)
enum : int32_t {
  ST_NOT_REACHED = 1,
  ST_NEWTON_FAIL = 2,
  ST_TANGENT = 4,
  ST_NOT_PD = 8,
  ST_NO_HIT = 16,
};

// crossing with transverse direction cosine below this is flagged TANGENT
constexpr double kTangentCos = 0.01;

// packed lower-triangle index, row-major: (i, j) -> i(i+1)/2 + j for j <= i
KF_HD constexpr int sym(int i, int j) { return i >= j ? (i * (i + 1)) / 2 + j : (j * (j + 1)) / 2 + i; }

KF_HD float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
KF_HD double fma_t(double a, double b, double c) { return fma(a, b, c); }

KF_HD float sqrt_t(float x) { return sqrtf(x); }
KF_HD double sqrt_t(double x) { return sqrt(x); }
KF_HD float log_t(float x) { return logf(x); }
KF_HD double log_t(double x) { return log(x); }
KF_HD float abs_t(float x) { return fabsf(x); }
KF_HD double abs_t(double x) { return fabs(x); }

// Reciprocal (correctly rounded) and a fast quotient for self-correcting
// steps (Newton updates); plain division on the host.
KF_HD float rcp_t(float x) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(x);
#else
  return 1.0f / x;
#endif
}
KF_HD double rcp_t(double x) { return 1.0 / x; }
KF_HD float div_fast(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
KF_HD double div_fast(double a, double b) { return a / b; }

// ---- masks and status words (one lane: bool and int32)
template <typename T>
struct Lanes {
  using M = bool;
  using I = int32_t;
  static constexpr bool kDouble = false;
};
template <>
struct Lanes<double> {
  using M = bool;
  using I = int32_t;
  static constexpr bool kDouble = true;
};

KF_HD bool any(bool m) { return m; }
KF_HD bool all(bool m) { return m; }
KF_HD float sel(bool m, float a, float b) { return m ? a : b; }
KF_HD double sel(bool m, double a, double b) { return m ? a : b; }
KF_HD int32_t set_bits(int32_t st, bool m, int32_t bits) { return m ? (st | bits) : st; }
KF_HD bool is_zero(int32_t st) { return st == 0; }
KF_HD int32_t zero_status(const int32_t*) { return 0; }

// sin(h)/h and cos(h).  Single precision: for |h| <= 1/2 the Taylor series
// 1 - h^2/3! + h^4/5! - h^6/7! + h^8/9!  and  1 - h^2/2! + ... - h^10/10!
// (alternating, so the truncation error is below the first omitted term:
// 2.5e-11 and 4e-13 at |h| = 1/2, far under float resolution); beyond that
// the library sincosf.  Double precision always uses the library sincos.
template <typename T>
KF_HD void sinc_cos_poly(T h, T& sch, T& ch) {
  const T h2 = h * h;
  sch = fma_t(h2, fma_t(h2, fma_t(h2, fma_t(h2, T(1.0f / 362880.0f), T(-1.0f / 5040.0f)), T(1.0f / 120.0f)),
                    T(-1.0f / 6.0f)),
              T(1.0f));
  ch = fma_t(
      h2,
      fma_t(h2, fma_t(h2, fma_t(h2, fma_t(h2, T(-1.0f / 3628800.0f), T(1.0f / 40320.0f)), T(-1.0f / 720.0f)),
                  T(1.0f / 24.0f)),
            T(-0.5f)),
      T(1.0f));
}
KF_HD void sinc_cos_lib(float h, float& sch, float& ch) {
  float sh;
  sincosf(h, &sh, &ch);
  sch = sh / h;
}
KF_HD void sinc_cos(float h, float& sch, float& ch) {
  if (fabsf(h) <= 0.5f)
    sinc_cos_poly(h, sch, ch);
  else
    sinc_cos_lib(h, sch, ch);
}
KF_HD void sinc_cos(double h, double& sch, double& ch) {
  double sh;
  sincos(h, &sh, &ch);
  const double h2 = h * h;
  sch = fabs(h) < 1e-4 ? 1.0 - h2 / 6.0 : sh / h;
}

// Error-free transformations (Knuth TwoSum, FMA TwoProd): a + b = s + e and
// a * b = p + e exactly in IEEE arithmetic.  Used to carry the position as an
// unevaluated pair hi + lo: a float32 position at r = 40 cm is only good to
// 1.9e-6 cm, which alone moves a chi2 of 30 by ~1e-3 at sigma = 0.01 cm.
template <typename T>
KF_HD void two_sum(T a, T b, T& s, T& e) {
  s = a + b;
  const T bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
template <typename T>
KF_HD void two_prod(T a, T b, T& p, T& e) {
  p = a * b;
  e = fma_t(a, b, -p);
}

// Helix displacement after path length s: dX, dY (relative to the start),
// momentum (PX, PY), sa = sin(th)/a, ca = (1-cos th)/a, cos th, sin th.
template <typename T>
struct HelixPoint {
  T dX, dY, PX, PY, sa, ca, cth, sth, th;
};

template <typename T>
KF_HD HelixPoint<T> helix_eval(T px, T py, T npx /* -px */, T k /*a/p*/, T ip /*1/p*/, T s) {
  HelixPoint<T> hp;
  const T th = k * s;
  const T h = T(0.5f) * th;
  T sch, ch;
  sinc_cos(h, sch, ch);
  const T sh = h * sch;
  const T sp = s * ip;
  hp.sa = (sp * sch) * ch;
  hp.ca = ((sp * h) * sch) * sch;
  const T tsh = sh + sh;
  hp.sth = tsh * ch;
  hp.cth = fma_t(-tsh, sh, T(1.0f));
  hp.th = th;
  hp.dX = fma_t(px, hp.sa, py * hp.ca);
  hp.dY = fma_t(npx, hp.ca, py * hp.sa);
  hp.PX = fma_t(px, hp.cth, py * hp.sth);
  hp.PY = fma_t(npx, hp.sth, py * hp.cth);
  return hp;
}

// Structural non-zeros of the transport Jacobian: J[i][l] may be non-zero
// for rows i < 5 and columns l != 2 (column z0 is e_z and row pz is e_pz,
// both handled apart).
KF_HD constexpr bool jnz(int i, int l) { return i < 5 && l != 2; }

// Propagate state p[6] (+ position low parts lo[3] when EXT) and packed
// covariance C[21], in place, to radius R, in the lanes of `live`.  Returns
// the status per lane (0 or an ST_* bit); a lane that fails, or is not live,
// is left unmodified.
template <typename T, int NEWTON, bool EXT>
KF_HD typename Lanes<T>::I propagate_lanes(T p[6], T lo[3], T C[21], T a, T R, typename Lanes<T>::M live) {
  using M = typename Lanes<T>::M;
  using I = typename Lanes<T>::I;
  I st = zero_status(static_cast<const I*>(nullptr));
  const T x = p[0], y = p[1], z = p[2], px = p[3], py = p[4], pz = p[5];
  const T npx = -px;
  const T xl = EXT ? lo[0] : T(0.0f), yl = EXT ? lo[1] : T(0.0f);
  const T pt2 = fma_t(px, px, py * py);
  const T pp2 = fma_t(pz, pz, pt2);
  const T pmag = sqrt_t(pp2);
  const T ip = rcp_t(pmag);
  const T pt = sqrt_t(pt2);
  const T ipt = rcp_t(pt);
  const T k = a * ip;
  // reachability: the transverse circle (centre x + py/a, y - px/a, radius
  // pT/|a|) reaches at most radius d + rho
  const T ia = rcp_t(a);
  const T cx = fma_t(py, ia, x), cy = fma_t(npx, ia, y);
  const T rho = pt * abs_t(ia);
  const T dctr = sqrt_t(fma_t(cx, cx, cy * cy));
  const M unreach = live & (R > dctr + rho);
  st = set_bits(st, unreach, ST_NOT_REACHED);
  const M run = live & !unreach;
  if (!any(run)) return st;
  // G0 = x^2 + y^2 - R^2 as an unevaluated pair (g0h + g0l)
  T g0h, g0l;
  {
    T a1, b1, a2, b2, a3, b3, s1, e1, s2, e2;
    two_prod(x, x, a1, b1);
    two_prod(y, y, a2, b2);
    two_prod(R, R, a3, b3);
    two_sum(a1, a2, s1, e1);
    two_sum(s1, -a3, s2, e2);
    g0h = s2;
    g0l = ((e1 + e2) + ((b1 + b2) - b3)) + T(2.0f) * fma_t(x, xl, y * yl);
  }
  // First guess from the transverse path t = s pT / p.  With u = pT/|pT|,
  // n = (uy, -ux) and kappa = a / pT the transverse displacement is
  // u sin(kappa t)/kappa + n (1 - cos(kappa t))/kappa, so
  //   g(t) = G0 + 2 b t + A t^2 - (kappa^2 t^3 / 12)(4 b + t) + O(kappa^3),
  // b = r0.u, A = 1 + kappa r0.n.  The quadratic's root, then one Newton
  // step on the polynomial for the cubic and quartic terms (its slope at the
  // root is 2 sqrt(disc)); the straight line (A = 1) where A is small, and no
  // polynomial step near a tangent crossing.  The guess is a few microns off
  // where the straight line is up to a millimetre off, so one Newton step
  // below usually meets the tolerance.
  const T tx = px * ipt, ty = py * ipt;
  const T b = fma_t(x, tx, y * ty);
  const T kap = a * ipt;
  T A = fma_t(kap, fma_t(x, ty, -(y * tx)), T(1.0f));
  A = sel(A > T(0.5f), A, T(1.0f));
  T disc = fma_t(b, b, -(A * (g0h + g0l)));
  disc = sel(disc > T(0.0f), disc, T(0.0f));
  const T sq = sqrt_t(disc);
  T t = (sq - b) * rcp_t(A);
  const T corr = (((kap * kap) * ((t * t) * t)) * fma_t(T(4.0f), b, t)) * (T(1.0f / 24.0f) * rcp_t(sq));
  t = sel(sq > fma_t(T(1e-3f), abs_t(b), T(1e-6f)), t + corr, t);
  T s = (t * pmag) * ipt;
  // Safeguarded Newton on g(s) = |r0 + d(s)|^2 - R^2 = G0 + 2 r0.d + |d|^2,
  // the large terms summed error-free when the position is a float pair.
  // [lo, hi] brackets the first crossing: g < 0 on the way out below it; a
  // point with g >= 0, or past the turning point (dg <= 0), bounds it from
  // above.  A step leaving the bracket is replaced by bisection.  Newton
  // converges quadratically (next error ~ ds^2 g''/2g'), so a lane stops
  // once ds^2 |p| <= tol (r.p): the remaining error is below the resolution
  // of the displacement.  Converged lanes are frozen.
  const T tol = T(Lanes<T>::kDouble ? 1e-20 : 1e-7);
  T lo_s = T(0.0f), hi_s = T(-1.0f);  // hi_s < 0: no upper bound yet
  M conv = !run;
  for (int it = 0; it < NEWTON; ++it) {
    if (all(conv)) break;
    const HelixPoint<T> hp = helix_eval(px, py, npx, k, ip, s);
    const T U = xl + hp.dX, W = yl + hp.dY;
    T g;
    if (EXT) {
      T h1, l1, h2, l2, s1, e1, s2, e2;
      two_prod(T(2.0f) * x, U, h1, l1);
      two_prod(T(2.0f) * y, W, h2, l2);
      two_sum(g0h, h1, s1, e1);
      two_sum(s1, h2, s2, e2);
      g = s2 + ((((g0l + l1) + l2) + (e1 + e2)) + fma_t(U, U, W * W));
    } else {
      g = g0h + ((g0l + T(2.0f) * fma_t(x, U, y * W)) + fma_t(U, U, W * W));
    }
    const T rp = fma_t(x + U, hp.PX, (y + W) * hp.PY);  // r.p at s
    const T dg = (T(2.0f) * rp) * ip;
    const M act = !conv;
    const M below = (g < T(0.0f)) & (dg > T(0.0f));
    lo_s = sel(act & below & (s > lo_s), s, lo_s);
    hi_s = sel(act & !below & ((hi_s < T(0.0f)) | (s < hi_s)), s, hi_s);
    T sn = sel(dg > T(0.0f), s - div_fast(g, dg), T(-1.0f));
    const M inb = (sn >= lo_s) & ((hi_s < T(0.0f)) | (sn <= hi_s));
    sn = sel(inb, sn, sel(hi_s >= T(0.0f), T(0.5f) * (lo_s + hi_s), T(2.0f) * s));
    const T ds = sn - s;
    s = sel(act, sn, s);
    conv = conv | (act & inb & ((ds * ds) * pmag <= tol * rp));
  }
  const HelixPoint<T> hp = helix_eval(px, py, npx, k, ip, s);
  const T X = x + (xl + hp.dX), Y = y + (yl + hp.dY);
  const T rdotp = fma_t(X, hp.PX, Y * hp.PY);
  // the crossing must be on the way out, and the solve converged: the
  // remaining Newton step |g| p / (2 r.p) below 1e-5 R
  const T gres = fma_t(X, X, fma_t(Y, Y, -(R * R)));
  const M out_bad = run & !((rdotp > T(0.0f)) & (s > T(0.0f)));
  st = set_bits(st, out_bad, ST_NOT_REACHED);
  M ok = run & !out_bad;
  const M unconv = ok & !(abs_t(gres) * pmag <= (T(2e-5f) * R) * rdotp);
  // no convergence: a layer at (or within rounding of) the largest radius of
  // the helix is not reached; anything else is a solver failure
  const M at_edge = unconv & (R > (dctr + rho) * T(1.0f - 1e-4f));
  st = set_bits(st, at_edge, ST_NOT_REACHED);
  st = set_bits(st, unconv & !at_edge, ST_NEWTON_FAIL);
  ok = ok & !unconv;
  const M tang = ok & (rdotp < (T(float(kTangentCos)) * R) * pt);
  st = set_bits(st, tang, ST_TANGENT);
  ok = ok & !tang;
  if (!any(ok)) return st;

  // ---- surface Jacobian
  // fixed-s partials D (rows x, y, z, px, py over columns px0, py0, pz0)
  const T ip2 = ip * ip;
  const T sp3 = (s * ip2) * ip;  // s / p^3
  const T thp2 = hp.th * ip2;    // theta / p^2
  const T P0[3] = {px, py, pz};
  const T nPXs = -(hp.PX * sp3), nPYs = -(hp.PY * sp3), nPZs = -(pz * sp3);
  const T nPYt = -(hp.PY * thp2), PXt = hp.PX * thp2;
  T D[5][3];
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    const T pk = P0[kk];
    D[0][kk] = kk == 2 ? nPXs * pk : fma_t(nPXs, pk, kk == 0 ? hp.sa : hp.ca);
    D[1][kk] = kk == 2 ? nPYs * pk : fma_t(nPYs, pk, kk == 0 ? -hp.ca : hp.sa);
    D[2][kk] = kk == 2 ? fma_t(nPZs, pk, s * ip) : nPZs * pk;
    D[3][kk] = kk == 2 ? nPYt * pk : fma_t(nPYt, pk, kk == 0 ? hp.cth : hp.sth);
    D[4][kk] = kk == 2 ? PXt * pk : fma_t(PXt, pk, kk == 0 ? -hp.sth : hp.cth);
  }
  // w_j = (dg/dx0_j)/(dg/ds) = (X dX/dx0_j + Y dY/dx0_j) p / (X PX + Y PY)
  const T irp = rcp_t(rdotp);
  const T iden = pmag * irp;
  T w[6];
  w[0] = X * iden;
  w[1] = Y * iden;
  w[2] = T(0.0f);
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) w[3 + kk] = fma_t(X, D[0][kk], Y * D[1][kk]) * iden;
  // -dF/ds
  const T nf[5] = {-(hp.PX * ip), -(hp.PY * ip), -(pz * ip), -(k * hp.PY), k * hp.PX};
  // J[i][l] for i < 5 over columns l in {0,1,3,4,5}; J[i][2] = (i == 2).
  // The transverse 2x2 corner is written in its cancellation-free form
  // (1 - PX X / r.p = Y PY / r.p, ...).
  T J[5][6];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    J[i][0] = nf[i] * w[0];
    J[i][1] = nf[i] * w[1];
    J[i][2] = T(0.0f);
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) J[i][3 + kk] = fma_t(nf[i], w[3 + kk], D[i][kk]);
  }
  J[0][0] = (Y * hp.PY) * irp;
  J[1][1] = (X * hp.PX) * irp;

  // ---- C' = J C J^T.  T1 = J C (rows 0..4); row 5 of J is e_pz.
  T T1[5][6];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
#pragma unroll
    for (int col = 0; col < 6; ++col) {
      T acc = (i == 2) ? C[sym(2, col)] : T(0.0f);
      bool first = i != 2;
#pragma unroll
      for (int l = 0; l < 6; ++l)
        if (jnz(i, l)) {
          acc = first ? J[i][l] * C[sym(l, col)] : fma_t(J[i][l], C[sym(l, col)], acc);
          first = false;
        }
      T1[i][col] = acc;
    }
  }
  T Cn[21];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T acc;
      if (j == 5) {
        acc = (i == 5) ? C[sym(5, 5)] : T1[i][5];
      } else if (i == 5) {
        // (J C J^T)_{5j} = (J C)_{j5}
        acc = T1[j][5];
      } else {
        acc = (j == 2) ? T1[i][2] : T(0.0f);
        bool first = j != 2;
#pragma unroll
        for (int l = 0; l < 6; ++l)
          if (jnz(j, l)) {
            acc = first ? T1[i][l] * J[j][l] : fma_t(T1[i][l], J[j][l], acc);
            first = false;
          }
      }
      Cn[sym(i, j)] = acc;
    }
  }
#pragma unroll
  for (int e = 0; e < 21; ++e) C[e] = sel(ok, Cn[e], C[e]);
  // new position: hi + lo, the displacement added error-free
  const T dZ = (pz * s) * ip;
  if (EXT) {
    T h, e;
    two_sum(x, hp.dX, h, e);
    T nh = h + (e + xl);
    lo[0] = sel(ok, (e + xl) - (nh - h), lo[0]);
    p[0] = sel(ok, nh, p[0]);
    two_sum(y, hp.dY, h, e);
    nh = h + (e + yl);
    lo[1] = sel(ok, (e + yl) - (nh - h), lo[1]);
    p[1] = sel(ok, nh, p[1]);
    two_sum(z, dZ, h, e);
    const T zl = lo[2];
    nh = h + (e + zl);
    lo[2] = sel(ok, (e + zl) - (nh - h), lo[2]);
    p[2] = sel(ok, nh, p[2]);
  } else {
    p[0] = sel(ok, X, p[0]);
    p[1] = sel(ok, Y, p[1]);
    p[2] = sel(ok, z + dZ, p[2]);
  }
  p[3] = sel(ok, hp.PX, p[3]);
  p[4] = sel(ok, hp.PY, p[4]);
  return st;
}

// One track (T = float or double): returns 0 or an ST_* bit.
template <typename T, int NEWTON, bool EXT>
KF_HD int propagate(T p[6], T lo[3], T C[21], T a, T R) {
  return propagate_lanes<T, NEWTON, EXT>(p, lo, C, a, R, true);
}

// Multiple scattering in a thin layer at the crossing just reached (Sec. 2:
// the KF folds the expected multiple scattering into the trajectory's
// uncertainty).  The direction turns by two independent projected angles of
// RMS theta0 in planes containing p, |p| unchanged: the momentum block gains
// theta0^2 (p^2 I - p p^T).  theta0 is the Highland formula with the
// Lynch-Dahl logarithm (Review of Particle Physics, passage of particles
// through matter) for a unit charge of mass `mass`:
//   theta0 = 0.0136 GeV / (beta p) sqrt(xe) (1 + 0.038 ln(xe / beta^2)),
// over xe = x_x0 / cos(incidence) radiation lengths, the incidence cosine
// being that of p with the cylinder normal (x, y, 0)/r; 1/(beta p)^2 = E^2/p^4.
template <typename T>
KF_HD void scatter(const T p[6], const T lo[3], T C[21], T x_x0, T mass) {
  const T X = p[0] + lo[0], Y = p[1] + lo[1];
  const T P[3] = {p[3], p[4], p[5]};
  const T p2 = fma_t(P[0], P[0], fma_t(P[1], P[1], P[2] * P[2]));
  const T cos_inc = abs_t(fma_t(X, P[0], Y * P[1])) / sqrt_t(fma_t(X, X, Y * Y) * p2);
  const T xe = x_x0 / (cos_inc > T(1e-6) ? cos_inc : T(1e-6));
  const T e2 = fma_t(mass, mass, p2);
  const T lg = fma_t(T(0.038), log_t(xe * (e2 / p2)), T(1.0));
  const T th2 = ((T(0.0136 * 0.0136) * xe) * (lg * lg)) * (e2 / (p2 * p2));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const T d = i == j ? fma_t(-P[i], P[j], p2) : -(P[i] * P[j]);
      C[sym(3 + i, 3 + j)] = fma_t(th2, d, C[sym(3 + i, 3 + j)]);
    }
}

// Residual r = m - H x with the position carried as hi + lo.
template <typename T, bool EXT>
KF_HD void residual(const T p[6], const T lo[3], T m0, T m1, T m2, T& r0, T& r1, T& r2) {
  r0 = (m0 - p[0]) - (EXT ? lo[0] : T(0.0f));
  r1 = (m1 - p[1]) - (EXT ? lo[1] : T(0.0f));
  r2 = (m2 - p[2]) - (EXT ? lo[2] : T(0.0f));
}

// S = C_pos + V (V diagonal), Si = S^-1 packed (00, 10, 11, 20, 21, 22), by
// the adjugate.  Returns the determinant.
template <typename T>
KF_HD T inverse_S(const T C[21], T v0, T v1, T v2, T Si[6]) {
  const T s00 = C[0] + v0, s10 = C[1], s11 = C[2] + v1, s20 = C[3], s21 = C[4], s22 = C[5] + v2;
  const T c00 = fma_t(s11, s22, -(s21 * s21));
  const T c10 = fma_t(s21, s20, -(s10 * s22));
  const T c20 = fma_t(s10, s21, -(s11 * s20));
  const T det = fma_t(s00, c00, fma_t(s10, c10, s20 * c20));
  const T id = rcp_t(det);
  Si[0] = c00 * id;
  Si[1] = c10 * id;
  Si[2] = fma_t(s00, s22, -(s20 * s20)) * id;
  Si[3] = c20 * id;
  Si[4] = fma_t(s20, s10, -(s00 * s21)) * id;
  Si[5] = fma_t(s00, s11, -(s10 * s10)) * id;
  return det;
}

// chi2 = r^T Si r, r = m - H x
template <typename T>
KF_HD T chi2_of(T r0, T r1, T r2, const T Si[6]) {
  const T u0 = fma_t(Si[0], r0, fma_t(Si[1], r1, Si[3] * r2));
  const T u1 = fma_t(Si[1], r0, fma_t(Si[2], r1, Si[4] * r2));
  const T u2 = fma_t(Si[3], r0, fma_t(Si[4], r1, Si[5] * r2));
  return fma_t(r0, u0, fma_t(r1, u1, r2 * u2));
}

// Kalman update with residual r (= m - H x'), Si = S^-1, V diagonal, in the
// lanes of `upd`:
//   K = C' H^T S^-1 (6x3),  x = x' + K r,
//   C = (I - K H) C' (I - K H)^T + K V K^T   (Joseph form; lower triangle kept).
// The gain is formed negated (nK = -K) so that every product below is one
// fused multiply-add.
template <typename T, bool EXT>
KF_HD void kalman_update_lanes(T p[6], T lo[3], T C[21], const T Si[6], T r0, T r1, T r2, T v0, T v1, T v2,
                               typename Lanes<T>::M upd) {
  const T nS0 = -Si[0], nS1 = -Si[1], nS2 = -Si[2], nS3 = -Si[3], nS4 = -Si[4], nS5 = -Si[5];
  T nK[6][3];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const T c0 = C[sym(i, 0)], c1 = C[sym(i, 1)], c2 = C[sym(i, 2)];
    nK[i][0] = fma_t(c0, nS0, fma_t(c1, nS1, c2 * nS3));
    nK[i][1] = fma_t(c0, nS1, fma_t(c1, nS2, c2 * nS4));
    nK[i][2] = fma_t(c0, nS3, fma_t(c1, nS4, c2 * nS5));
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const T ndx = fma_t(nK[i][0], r0, fma_t(nK[i][1], r1, nK[i][2] * r2));  // -(K r)_i
    if (EXT && i < 3) {
      T h, e;
      two_sum(p[i], lo[i] - ndx, h, e);
      p[i] = sel(upd, h, p[i]);
      lo[i] = sel(upd, e, lo[i]);
    } else {
      p[i] = sel(upd, p[i] - ndx, p[i]);
    }
  }
  // B = (I - K H) C'  (full 6x6)
  T B[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j)
      B[i][j] = fma_t(nK[i][0], C[sym(0, j)],
                      fma_t(nK[i][1], C[sym(1, j)], fma_t(nK[i][2], C[sym(2, j)], C[sym(i, j)])));
  // C = B (I - K H)^T + K V K^T, with K V K^T = (nK V) nK^T
  const T v[3] = {v0, v1, v2};
  T nKV[6][3];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) nKV[i][kk] = nK[i][kk] * v[kk];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T acc = B[i][j];
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) acc = fma_t(nKV[i][kk], nK[j][kk], acc);
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) acc = fma_t(B[i][kk], nK[j][kk], acc);
      C[sym(i, j)] = sel(upd, acc, C[sym(i, j)]);
    }
}

template <typename T, bool EXT>
KF_HD void kalman_update(T p[6], T lo[3], T C[21], const T Si[6], T r0, T r1, T r2, T v0, T v1, T v2) {
  kalman_update_lanes<T, EXT>(p, lo, C, Si, r0, r1, r2, v0, v1, v2, true);
}

// Mixed precision: the same update with S^-1, the gain and the Joseph
// covariance downdate in FP64 (inputs and outputs stay float; the position
// correction is added to the hi + lo pair).  Returns the chi2 increment.
KF_HD float kalman_update_f64(float p[6], float lo[3], float C[21], float r0, float r1, float r2, float v0, float v1,
                              float v2) {
  double Cd[21];
#pragma unroll
  for (int e = 0; e < 21; ++e) Cd[e] = C[e];
  double Si[6];
  inverse_S<double>(Cd, v0, v1, v2, Si);
  const double c2 = chi2_of<double>(r0, r1, r2, Si);
  double dx[6] = {0, 0, 0, 0, 0, 0}, dlo[3] = {0, 0, 0};
  kalman_update<double, false>(dx, dlo, Cd, Si, r0, r1, r2, v0, v1, v2);
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (i < 3) {
      float h, e;
      two_sum(p[i], lo[i] + float(dx[i]), h, e);
      p[i] = h;
      lo[i] = e;
    } else {
      p[i] = p[i] + float(dx[i]);
    }
  }
#pragma unroll
  for (int e = 0; e < 21; ++e) C[e] = float(Cd[e]);
  return float(c2);
}

}  // namespace kf
