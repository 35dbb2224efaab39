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
// State (x, y, z, px, py, pz) in cm and GeV; a = q * 0.00299792458 * Bz.
// Helix:  theta = a s / p,
//   x(s)  = x0 + px0 sin(th)/a + py0 (1 - cos th)/a
//   y(s)  = y0 + py0 sin(th)/a - px0 (1 - cos th)/a,   z(s) = z0 + pz0 s / p
//   px(s) = px0 cos th + py0 sin th,   py(s) = py0 cos th - px0 sin th.
// sin(th)/a = (s/p) sinc(h) cos(h) and (1 - cos th)/a = (s/p) h sinc(h)^2
// with h = th/2: no 1/a and no 1 - cos cancellation.
// The path length s to radius R solves g(s) = x(s)^2 + y(s)^2 - R^2 = 0 by
// Newton iterations from the straight-line guess.  The transport Jacobian is
// the surface one, J = dF/dx0|_s - (dF/ds)(dg/dx0|_s)/(dg/ds).
//
// Templated on the arithmetic type T (float for the batched path, double for
// the plain per-event form).  Compiles for the host too (no CUDA intrinsics)
// so that the same source can be exercised off the GPU.
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

KF_HD float sqrt_t(float x) { return sqrtf(x); }
KF_HD double sqrt_t(double x) { return sqrt(x); }
KF_HD float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
KF_HD double fma_t(double a, double b, double c) { return fma(a, b, c); }
KF_HD float abs_t(float x) { return fabsf(x); }
KF_HD double abs_t(double x) { return fabs(x); }

// Reciprocal (correctly rounded) and a fast quotient for self-correcting
// steps (Newton updates, Jacobian-only terms); plain division on the host.
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

// sin(h)/h and cos(h).  Single precision: for |h| <= 1/2 the Taylor series
// 1 - h^2/3! + h^4/5! - h^6/7! + h^8/9!  and  1 - h^2/2! + ... - h^10/10!
// (alternating, so the truncation error is below the first omitted term:
// 2.5e-11 and 4e-13 at |h| = 1/2, far under float resolution); beyond that
// the library sincosf.  Double precision always uses the library sincos.
KF_HD void sinc_cos(float h, float& sch, float& ch) {
  if (fabsf(h) <= 0.5f) {
    const float h2 = h * h;
    sch = fmaf(h2, fmaf(h2, fmaf(h2, fmaf(h2, 1.0f / 362880.0f, -1.0f / 5040.0f), 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
    ch = fmaf(h2,
              fmaf(h2, fmaf(h2, fmaf(h2, fmaf(h2, -1.0f / 3628800.0f, 1.0f / 40320.0f), -1.0f / 720.0f), 1.0f / 24.0f),
                   -0.5f),
              1.0f);
  } else {
    float sh;
    sincosf(h, &sh, &ch);
    sch = sh / h;
  }
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
KF_HD HelixPoint<T> helix_eval(T px, T py, T k /*a/p*/, T ip /*1/p*/, T s) {
  HelixPoint<T> hp;
  const T th = k * s;
  const T h = T(0.5) * th;
  T sch, ch;
  sinc_cos(h, sch, ch);
  const T sh = h * sch;
  const T sp = s * ip;
  hp.sa = sp * sch * ch;
  hp.ca = sp * h * sch * sch;
  hp.sth = T(2) * sh * ch;
  hp.cth = T(1) - T(2) * sh * sh;
  hp.th = th;
  hp.dX = px * hp.sa + py * hp.ca;
  hp.dY = py * hp.sa - px * hp.ca;
  hp.PX = px * hp.cth + py * hp.sth;
  hp.PY = py * hp.cth - px * hp.sth;
  return hp;
}

// Structural non-zeros of the transport Jacobian: J[i][l] may be non-zero
// for rows i < 5 and columns l != 2 (column z0 is e_z and row pz is e_pz,
// both handled apart).
KF_HD constexpr bool jnz(int i, int l) { return i < 5 && l != 2; }

// Propagate state p[6] (+ position low parts lo[3] when EXT) and packed
// covariance C[21], in place, to radius R.  Returns 0 or an ST_* bit; on
// failure nothing is modified.
template <typename T, int NEWTON, bool EXT>
KF_HD int propagate(T p[6], T lo[3], T C[21], T a, T R) {
  const T x = p[0], y = p[1], z = p[2], px = p[3], py = p[4], pz = p[5];
  const T xl = EXT ? lo[0] : T(0), yl = EXT ? lo[1] : T(0);
  const T pt2 = px * px + py * py;
  const T pp2 = pt2 + pz * pz;
  const T pmag = sqrt_t(pp2);
  const T ip = rcp_t(pmag);
  const T ipt = rcp_t(sqrt_t(pt2));
  const T k = a * ip;
  // reachability: the transverse circle (centre x + py/a, y - px/a, radius
  // pT/|a|) reaches at most radius d + rho
  if (a != T(0)) {
    const T ia = rcp_t(a);
    const T cx = x + py * ia, cy = y - px * ia;
    const T rho = sqrt_t(pt2) * abs_t(ia);
    if (R > sqrt_t(cx * cx + cy * cy) + rho) return ST_NOT_REACHED;
  }
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
    g0l = (e1 + e2) + (b1 + b2 - b3) + T(2) * (x * xl + y * yl);
  }
  // straight-line first guess in the transverse plane
  const T tx = px * ipt, ty = py * ipt;
  const T b = x * tx + y * ty;
  T disc = b * b - (g0h + g0l);
  disc = disc > T(0) ? disc : T(0);
  T s = (sqrt_t(disc) - b) * pmag * ipt;
  // Safeguarded Newton on g(s) = |r0 + d(s)|^2 - R^2 = G0 + 2 r0.d + |d|^2,
  // the large terms summed error-free when the position is a float pair.
  // [lo, hi] brackets the first crossing: g < 0 on the way out below it; a
  // point with g >= 0, or past the turning point (dg <= 0), bounds it from
  // above.  A step leaving the bracket is replaced by bisection.  Newton
  // converges quadratically (next error ~ ds^2 g''/2g'), so the loop stops
  // once ds^2 |p| <= 1e-7 (r.p): the remaining error is below float
  // resolution of the displacement.
  T lo_s = T(0), hi_s = T(-1);  // hi_s < 0: no upper bound yet
  for (int it = 0; it < NEWTON; ++it) {
    const HelixPoint<T> hp = helix_eval(px, py, k, ip, s);
    const T U = xl + hp.dX, W = yl + hp.dY;
    T g;
    if (EXT) {
      T h1, l1, h2, l2, s1, e1, s2, e2;
      two_prod(T(2) * x, U, h1, l1);
      two_prod(T(2) * y, W, h2, l2);
      two_sum(g0h, h1, s1, e1);
      two_sum(s1, h2, s2, e2);
      g = s2 + ((g0l + l1 + l2 + e1 + e2) + (U * U + W * W));
    } else {
      g = g0h + (g0l + T(2) * (x * U + y * W) + (U * U + W * W));
    }
    const T rp = (x + U) * hp.PX + (y + W) * hp.PY;  // r.p at s
    const T dg = T(2) * rp * ip;
    if (g < T(0) && dg > T(0)) {
      lo_s = s > lo_s ? s : lo_s;
    } else {
      hi_s = (hi_s < T(0) || s < hi_s) ? s : hi_s;
    }
    T sn = dg > T(0) ? s - div_fast(g, dg) : T(-1);
    const bool in_bracket = sn >= lo_s && (hi_s < T(0) || sn <= hi_s);
    if (!in_bracket) sn = hi_s >= T(0) ? T(0.5) * (lo_s + hi_s) : T(2) * s;
    const T ds = sn - s;
    s = sn;
    if (in_bracket && ds * ds * pmag <= (sizeof(T) == 4 ? T(1e-7) : T(1e-20)) * rp) break;
  }
  const HelixPoint<T> hp = helix_eval(px, py, k, ip, s);
  const T X = x + (xl + hp.dX), Y = y + (yl + hp.dY);
  const T rdotp = X * hp.PX + Y * hp.PY;
  // the crossing must be on the way out, and the solve converged: the
  // remaining Newton step |g| p / (2 r.p) below 1e-5 R
  const T gres = X * X + Y * Y - R * R;
  if (!(rdotp > T(0)) || !(s > T(0))) return ST_NOT_REACHED;
  if (!(abs_t(gres) * pmag <= T(2e-5) * R * rdotp)) {
    // no convergence: a layer at (or within rounding of) the largest radius
    // of the helix is not reached; anything else is a solver failure
    if (a != T(0)) {
      const T ia = T(1) / a;
      const T cx = x + py * ia, cy = y - px * ia;
      if (R > (sqrt_t(cx * cx + cy * cy) + sqrt_t(pt2) * abs_t(ia)) * (T(1) - T(1e-4))) return ST_NOT_REACHED;
    }
    return ST_NEWTON_FAIL;
  }
  if (rdotp < T(kTangentCos) * R * sqrt_t(pt2)) return ST_TANGENT;

  // ---- surface Jacobian
  // fixed-s partials D (rows x, y, z, px, py over columns px0, py0, pz0)
  const T ip2 = ip * ip;
  const T sp3 = s * ip2 * ip;  // s / p^3
  const T thp2 = hp.th * ip2;  // theta / p^2
  const T P0[3] = {px, py, pz};
  T D[5][3];
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    const T pk = P0[kk];
    D[0][kk] = (kk == 0 ? hp.sa : kk == 1 ? hp.ca : T(0)) - hp.PX * sp3 * pk;
    D[1][kk] = (kk == 0 ? -hp.ca : kk == 1 ? hp.sa : T(0)) - hp.PY * sp3 * pk;
    D[2][kk] = (kk == 2 ? s * ip : T(0)) - pz * sp3 * pk;
    D[3][kk] = (kk == 0 ? hp.cth : kk == 1 ? hp.sth : T(0)) - hp.PY * thp2 * pk;
    D[4][kk] = (kk == 0 ? -hp.sth : kk == 1 ? hp.cth : T(0)) + hp.PX * thp2 * pk;
  }
  // w_j = (dg/dx0_j)/(dg/ds) = (X dX/dx0_j + Y dY/dx0_j) p / (X PX + Y PY)
  const T irp = rcp_t(rdotp);
  const T iden = pmag * irp;
  T w[6];
  w[0] = X * iden;
  w[1] = Y * iden;
  w[2] = T(0);
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) w[3 + kk] = (X * D[0][kk] + Y * D[1][kk]) * iden;
  // dF/ds
  const T f[5] = {hp.PX * ip, hp.PY * ip, pz * ip, k * hp.PY, -k * hp.PX};
  // J[i][l] for i < 5 over columns l in {0,1,3,4,5}; J[i][2] = (i == 2).
  // The transverse 2x2 corner is written in its cancellation-free form
  // (1 - PX X / r.p = Y PY / r.p, ...).
  T J[5][6];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    J[i][0] = -f[i] * w[0];
    J[i][1] = -f[i] * w[1];
    J[i][2] = T(0);
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) J[i][3 + kk] = D[i][kk] - f[i] * w[3 + kk];
  }
  J[0][0] = Y * hp.PY * irp;
  J[1][1] = X * hp.PX * irp;

  // ---- C' = J C J^T.  T1 = J C (rows 0..4); row 5 of J is e_pz.
  T T1[5][6];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
#pragma unroll
    for (int col = 0; col < 6; ++col) {
      T acc = (i == 2) ? C[sym(2, col)] : T(0);
#pragma unroll
      for (int l = 0; l < 6; ++l)
        if (jnz(i, l)) acc = fma_t(J[i][l], C[sym(l, col)], acc);
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
        acc = (j == 2) ? T1[i][2] : T(0);
#pragma unroll
        for (int l = 0; l < 6; ++l)
          if (jnz(j, l)) acc = fma_t(T1[i][l], J[j][l], acc);
      }
      Cn[sym(i, j)] = acc;
    }
  }
#pragma unroll
  for (int e = 0; e < 21; ++e) C[e] = Cn[e];
  // new position: hi + lo, the displacement added error-free
  const T dZ = pz * s * ip;
  if (EXT) {
    T h, e;
    two_sum(x, hp.dX, h, e);
    p[0] = h + (e + xl);
    lo[0] = (e + xl) - (p[0] - h);
    two_sum(y, hp.dY, h, e);
    p[1] = h + (e + yl);
    lo[1] = (e + yl) - (p[1] - h);
    two_sum(z, dZ, h, e);
    const T zl = lo[2];
    p[2] = h + (e + zl);
    lo[2] = (e + zl) - (p[2] - h);
  } else {
    p[0] = X;
    p[1] = Y;
    p[2] = z + dZ;
  }
  p[3] = hp.PX;
  p[4] = hp.PY;
  return 0;
}

// Residual r = m - H x with the position carried as hi + lo.
template <typename T, bool EXT>
KF_HD void residual(const T p[6], const T lo[3], T m0, T m1, T m2, T& r0, T& r1, T& r2) {
  r0 = (m0 - p[0]) - (EXT ? lo[0] : T(0));
  r1 = (m1 - p[1]) - (EXT ? lo[1] : T(0));
  r2 = (m2 - p[2]) - (EXT ? lo[2] : T(0));
}

// S = C_pos + V (V diagonal), Si = S^-1 packed (00, 10, 11, 20, 21, 22), by
// the adjugate.  Returns the determinant.
template <typename T>
KF_HD T inverse_S(const T C[21], T v0, T v1, T v2, T Si[6]) {
  const T s00 = C[0] + v0, s10 = C[1], s11 = C[2] + v1, s20 = C[3], s21 = C[4], s22 = C[5] + v2;
  const T c00 = s11 * s22 - s21 * s21;
  const T c10 = s21 * s20 - s10 * s22;
  const T c20 = s10 * s21 - s11 * s20;
  const T det = s00 * c00 + s10 * c10 + s20 * c20;
  const T id = rcp_t(det);
  Si[0] = c00 * id;
  Si[1] = c10 * id;
  Si[2] = (s00 * s22 - s20 * s20) * id;
  Si[3] = c20 * id;
  Si[4] = (s20 * s10 - s00 * s21) * id;
  Si[5] = (s00 * s11 - s10 * s10) * id;
  return det;
}

// chi2 = r^T Si r, r = m - H x
template <typename T>
KF_HD T chi2_of(T r0, T r1, T r2, const T Si[6]) {
  const T u0 = Si[0] * r0 + Si[1] * r1 + Si[3] * r2;
  const T u1 = Si[1] * r0 + Si[2] * r1 + Si[4] * r2;
  const T u2 = Si[3] * r0 + Si[4] * r1 + Si[5] * r2;
  return r0 * u0 + r1 * u1 + r2 * u2;
}

// Kalman update with residual r (= m - H x'), Si = S^-1, V diagonal:
//   K = C' H^T S^-1 (6x3),  x = x' + K r,
//   C = (I - K H) C' (I - K H)^T + K V K^T   (Joseph form; lower triangle kept).
template <typename T, bool EXT>
KF_HD void kalman_update(T p[6], T lo[3], T C[21], const T Si[6], T r0, T r1, T r2, T v0, T v1, T v2) {
  T K[6][3];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const T c0 = C[sym(i, 0)], c1 = C[sym(i, 1)], c2 = C[sym(i, 2)];
    K[i][0] = c0 * Si[0] + c1 * Si[1] + c2 * Si[3];
    K[i][1] = c0 * Si[1] + c1 * Si[2] + c2 * Si[4];
    K[i][2] = c0 * Si[3] + c1 * Si[4] + c2 * Si[5];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const T dx = K[i][0] * r0 + K[i][1] * r1 + K[i][2] * r2;
    if (EXT && i < 3) {
      T h, e;
      two_sum(p[i], lo[i] + dx, h, e);
      p[i] = h;
      lo[i] = e;
    } else {
      p[i] = p[i] + dx;
    }
  }
  // B = (I - K H) C'  (full 6x6)
  T B[6][6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j)
      B[i][j] = C[sym(i, j)] - (K[i][0] * C[sym(0, j)] + K[i][1] * C[sym(1, j)] + K[i][2] * C[sym(2, j)]);
  const T v[3] = {v0, v1, v2};
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      T acc = B[i][j] - (B[i][0] * K[j][0] + B[i][1] * K[j][1] + B[i][2] * K[j][2]);
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) acc = fma_t(K[i][kk] * v[kk], K[j][kk], acc);
      C[sym(i, j)] = acc;
    }
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
