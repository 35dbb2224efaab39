/*
 * kf_oracle.c -- plain, slow FP64 reference ("oracle") of the Kalman-filter
 * track fit and combinatorial track building of Cerati et al., "Kalman Filter
 * Tracking on Parallel Architectures" (CTD2016), Sec. 2 (KF tracking, the
 * fit) and Sec. 3 (track building, best-hit and clone-engine selection).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle for the CUDA
 * library.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * The paper defers the filter mathematics to Fruhwirth (1987) and prints no
 * formula; what follows is the textbook extended Kalman filter for a helix in
 * a uniform solenoidal field, written out step by step in the filter's own
 * order (propagate -> transport covariance -> residual, chi2 -> gain ->
 * update), with every matrix stored full (6x6, row-major) and every loop
 * plain.  No blocking, fusion or sparsity tricks.
 *
 * Units: cm, GeV, tesla.  State x = (x, y, z, px, py, pz).
 * a = q * C_LIGHT * Bz (GeV/cm, signed); theta = a s / p for path length s.
 *
 * Parity status of each function (what pins it, see tests/test_oracle_*.py):
 *   orc_helix_at            pinned: |p| and pT conservation, B->0 straight line,
 *                           closed-form circle, ODE residual.
 *   orc_path_length_*       pinned: closed-form circle vs Newton, independent
 *                           turning-angle formula for tracks from the origin.
 *   orc_propagate (J)       pinned: central finite differences of the full
 *                           propagate-to-radius map.
 *   orc_update              pinned: Joseph == standard form; zero-distance
 *                           information-form identity; chi2(3) statistics and
 *                           unit pulls on correctly smeared hits.
 *   orc_fit                 pinned: noise-free fit recovers truth, chi2 = 0.
 *   orc_build               pinned: exhaustive enumeration on tiny inputs.
 *   orc_scattering_q        pinned: symmetric, rank 2 with p in its null space,
 *                           trace 2 p^2 theta0^2 with theta0 from a golden table
 *                           of the Highland formula (40-digit mpmath, written
 *                           without this file or the generator); fits of tracks simulated
 *                           with scattering kinks have chi2 mean 3 and unit
 *                           pulls in every eta range (the incidence factor).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_C_LIGHT 0.00299792458 /* GeV / (T cm) */

/* per-track status bits (same meaning as the library's) */
#define ORC_NOT_REACHED 1 /* the helix never reaches the layer radius      */
#define ORC_NEWTON_FAIL 2 /* path-length solve did not converge           */
#define ORC_TANGENT 4     /* crossing within 0.01 (cosine) of tangent      */
#define ORC_NOT_PD 8      /* final 5x5 projected covariance not PD          */
#define ORC_NO_HIT 16     /* at least one layer without a hit              */

#define ORC_TANGENT_COS 0.01

/* ------------------------------------------------------------------------ */
/* small helpers                                                              */

static double sinc(double t) /* sin(t)/t, exact limit 1 at t = 0 */
{
    if (fabs(t) < 1e-4) return 1.0 - t * t / 6.0;
    return sin(t) / t;
}

static void mat6_mul(const double *A, const double *B, double *C) /* C = A B */
{
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 6; ++k) acc += A[i * 6 + k] * B[k * 6 + j];
            C[i * 6 + j] = acc;
        }
}

static void mat6_transpose(const double *A, double *T)
{
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) T[j * 6 + i] = A[i * 6 + j];
}

/* inverse of a 3x3 matrix by the adjugate; returns the determinant */
static double mat3_inv(const double *S, double *Si)
{
    double c00 = S[4] * S[8] - S[5] * S[7];
    double c01 = S[5] * S[6] - S[3] * S[8];
    double c02 = S[3] * S[7] - S[4] * S[6];
    double det = S[0] * c00 + S[1] * c01 + S[2] * c02;
    double id = 1.0 / det;
    Si[0] = c00 * id;
    Si[1] = (S[2] * S[7] - S[1] * S[8]) * id;
    Si[2] = (S[1] * S[5] - S[2] * S[4]) * id;
    Si[3] = c01 * id;
    Si[4] = (S[0] * S[8] - S[2] * S[6]) * id;
    Si[5] = (S[2] * S[3] - S[0] * S[5]) * id;
    Si[6] = c02 * id;
    Si[7] = (S[1] * S[6] - S[0] * S[7]) * id;
    Si[8] = (S[0] * S[4] - S[1] * S[3]) * id;
    return det;
}

/* ------------------------------------------------------------------------ */
/* helix in a uniform field Bz                                                */

/* State after path length s.  Momentum rotates by theta = a s / p:
 *   px = px0 cos(th) + py0 sin(th),  py = py0 cos(th) - px0 sin(th),
 *   x  = x0 + (px0 sin(th) + py0 (1 - cos(th))) / a,
 *   y  = y0 + (py0 sin(th) - px0 (1 - cos(th))) / a,
 *   z  = z0 + pz0 s / p.
 * sin(th)/a and (1-cos(th))/a are written as (s/p) sinc(th) and
 * (s/p)(th/2) sinc^2(th/2): the same values, without the 1/a singularity. */
void orc_helix_at(const double *x0, double a, double s, double *out)
{
    double p = sqrt(x0[3] * x0[3] + x0[4] * x0[4] + x0[5] * x0[5]);
    double th = a * s / p;
    double sa = (s / p) * sinc(th);                                 /* sin(th)/a     */
    double ca = (s / p) * (0.5 * th) * sinc(0.5 * th) * sinc(0.5 * th); /* (1-cos th)/a */
    double c = cos(th), sn = sin(th);
    out[0] = x0[0] + x0[3] * sa + x0[4] * ca;
    out[1] = x0[1] + x0[4] * sa - x0[3] * ca;
    out[2] = x0[2] + x0[5] * s / p;
    out[3] = x0[3] * c + x0[4] * sn;
    out[4] = x0[4] * c - x0[3] * sn;
    out[5] = x0[5];
}

/* g(s) = x(s)^2 + y(s)^2 - R^2 and dg/ds = 2 (x px + y py) / p */
static void radius_residual(const double *x0, double a, double R, double s, double *g,
                            double *dg)
{
    double st[6];
    orc_helix_at(x0, a, s, st);
    double p = sqrt(x0[3] * x0[3] + x0[4] * x0[4] + x0[5] * x0[5]);
    *g = st[0] * st[0] + st[1] * st[1] - R * R;
    *dg = 2.0 * (st[0] * st[3] + st[1] * st[4]) / p;
}

/* Closed form: the transverse circle (centre c = (x0 + py0/a, y0 - px0/a),
 * radius rho = pT/|a|) meets r = R where c.u = (R^2 - d^2 - rho^2)/(2 rho),
 * u the unit vector from c.  Of the two crossings the one reached first along
 * the motion (clockwise for a > 0) is taken.  Returns 0 or ORC_NOT_REACHED. */
int orc_path_length_circle(const double *x0, double a, double R, double *s_out)
{
    double px = x0[3], py = x0[4], pz = x0[5];
    double pt = sqrt(px * px + py * py);
    double p = sqrt(pt * pt + pz * pz);
    if (pt <= 0.0 || a == 0.0) return ORC_NOT_REACHED;
    double rho = pt / fabs(a);
    double cx = x0[0] + py / a, cy = x0[1] - px / a;
    double d = sqrt(cx * cx + cy * cy);
    double kap = (R * R - d * d - rho * rho) / (2.0 * rho * d);
    if (!(kap >= -1.0 && kap <= 1.0)) return ORC_NOT_REACHED;
    double psic = atan2(cy, cx), alpha = acos(kap);
    double psi0 = atan2(x0[1] - cy, x0[0] - cx);
    double best = INFINITY;
    for (int k = 0; k < 2; ++k) {
        double psit = psic + (k == 0 ? alpha : -alpha);
        double tau = (a > 0) ? (psi0 - psit) : (psit - psi0);
        tau = fmod(tau, 2.0 * M_PI);
        if (tau < 0) tau += 2.0 * M_PI;
        if (tau < best) best = tau;
    }
    *s_out = best * rho * p / pt;
    return 0;
}

/* Newton iteration on g(s) from s_start; stops when |ds| < tol. */
int orc_path_length_newton(const double *x0, double a, double R, double s_start, double tol,
                           int max_iter, double *s_out, int *iters)
{
    double s = s_start;
    for (int it = 0; it < max_iter; ++it) {
        double g, dg;
        radius_residual(x0, a, R, s, &g, &dg);
        if (dg == 0.0) {
            *s_out = s;
            *iters = it;
            return ORC_NEWTON_FAIL;
        }
        double ds = -g / dg;
        s += ds;
        if (fabs(ds) < tol) {
            *s_out = s;
            *iters = it + 1;
            return 0;
        }
    }
    *s_out = s;
    *iters = max_iter;
    return ORC_NEWTON_FAIL;
}

/* Straight-line first guess: the transverse line from (x0, y0) along
 * (px0, py0) meets r = R after transverse distance u; s = u p / pT. */
double orc_straight_line_guess(const double *x0, double R)
{
    double pt = sqrt(x0[3] * x0[3] + x0[4] * x0[4]);
    double p = sqrt(pt * pt + x0[5] * x0[5]);
    double tx = x0[3] / pt, ty = x0[4] / pt;
    double b = x0[0] * tx + x0[1] * ty;
    double c = x0[0] * x0[0] + x0[1] * x0[1] - R * R;
    double disc = b * b - c;
    if (disc < 0) disc = 0;
    double u = -b + sqrt(disc);
    return u * p / pt;
}

/* Propagate to the cylinder r = R: path length (closed form, polished by
 * Newton to |ds| < 1e-13 cm), the new state, and the transport Jacobian
 *     J = dF/dx0 |_s + (dF/ds) (ds/dx0)^T,   ds/dx0 = -(dg/dx0 |_s) / (dg/ds),
 * with theta depending on p0 through p (d theta / d p_i = -theta p_i / p^2). */
int orc_propagate(const double *x0, double a, double R, double *x1, double *J, double *s_out)
{
    double s;
    int st = orc_path_length_circle(x0, a, R, &s);
    if (st) return st;
    int it;
    double s2;
    if (orc_path_length_newton(x0, a, R, s, 1e-13, 50, &s2, &it) == 0) s = s2;

    double px0 = x0[3], py0 = x0[4], pz0 = x0[5];
    double p2 = px0 * px0 + py0 * py0 + pz0 * pz0, p = sqrt(p2), pt = sqrt(px0 * px0 + py0 * py0);
    orc_helix_at(x0, a, s, x1);
    double xx = x1[0], yy = x1[1], px = x1[3], py = x1[4];
    double dgds = 2.0 * (xx * px + yy * py) / p;
    if (dgds <= 0.0) return ORC_NOT_REACHED; /* would cross inwards */
    if ((xx * px + yy * py) / (R * pt) < ORC_TANGENT_COS) return ORC_TANGENT;

    double th = a * s / p;
    double sa = (s / p) * sinc(th);
    double ca = (s / p) * (0.5 * th) * sinc(0.5 * th) * sinc(0.5 * th);
    double c = cos(th), sn = sin(th);
    double dth[3] = {-th * px0 / p2, -th * py0 / p2, -th * pz0 / p2}; /* d theta/d p0 */

    /* fixed-s partial derivatives dF/dx0 */
    double D[36];
    memset(D, 0, sizeof D);
    D[0 * 6 + 0] = 1.0;
    D[1 * 6 + 1] = 1.0;
    D[2 * 6 + 2] = 1.0;
    D[5 * 6 + 5] = 1.0;
    for (int k = 0; k < 3; ++k) {
        int col = 3 + k;
        /* x: explicit terms + (px/a) dtheta/dp_k, where (px/a) dtheta = -px s p_k/p^3 */
        double expl_x = (k == 0) ? sa : (k == 1) ? ca : 0.0;
        double expl_y = (k == 0) ? -ca : (k == 1) ? sa : 0.0;
        double pk = x0[3 + k];
        D[0 * 6 + col] = expl_x - px * s * pk / (p2 * p);
        D[1 * 6 + col] = expl_y - py * s * pk / (p2 * p);
        D[2 * 6 + col] = ((k == 2) ? s / p : 0.0) - pz0 * s * pk / (p2 * p);
        double expl_px = (k == 0) ? c : (k == 1) ? sn : 0.0;
        double expl_py = (k == 0) ? -sn : (k == 1) ? c : 0.0;
        D[3 * 6 + col] = expl_px + py * dth[k];
        D[4 * 6 + col] = expl_py - px * dth[k];
    }
    /* dF/ds */
    double dFds[6] = {px / p, py / p, pz0 / p, a * py / p, -a * px / p, 0.0};
    /* dg/dx0 at fixed s = 2 x dx/dx0 + 2 y dy/dx0 */
    double dgdx0[6];
    for (int j = 0; j < 6; ++j) dgdx0[j] = 2.0 * xx * D[0 * 6 + j] + 2.0 * yy * D[1 * 6 + j];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) J[i * 6 + j] = D[i * 6 + j] - dFds[i] * dgdx0[j] / dgds;
    if (s_out) *s_out = s;
    return 0;
}

/* Multiple scattering in a thin layer at the crossing state x (Sec. 2: the KF
 * folds the expected multiple scattering into the trajectory's uncertainty):
 * the direction turns by two independent projected angles of RMS theta0 in
 * planes containing p, |p| unchanged, so the momentum block of the process
 * noise is theta0^2 (p^2 I - p p^T) and every other block is zero.  theta0 is
 * the Highland formula with the Lynch-Dahl logarithm (Review of Particle
 * Physics, passage of particles through matter) for a unit charge of mass
 * `mass` (GeV) over the path x_x0 / cos(incidence) radiation lengths, the
 * incidence cosine being that of p with the cylinder normal (x, y, 0)/r:
 *   theta0 = 0.0136 GeV / (beta p) sqrt(xe) (1 + 0.038 ln(xe / beta^2)). */
void orc_scattering_q(const double *x, double x_x0, double mass, double *Q)
{
    const double px = x[3], py = x[4], pz = x[5];
    const double p2 = px * px + py * py + pz * pz, p = sqrt(p2);
    const double r = sqrt(x[0] * x[0] + x[1] * x[1]);
    const double cos_inc = fabs(x[0] * px + x[1] * py) / (r * p);
    const double xe = x_x0 / (cos_inc > 1e-6 ? cos_inc : 1e-6);
    const double beta2 = p2 / (p2 + mass * mass);
    const double th0 = 0.0136 / (sqrt(beta2) * p) * sqrt(xe) * (1.0 + 0.038 * log(xe / beta2));
    const double P[3] = {px, py, pz};
    for (int i = 0; i < 36; ++i) Q[i] = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Q[(3 + i) * 6 + 3 + j] = th0 * th0 * ((i == j ? p2 : 0.0) - P[i] * P[j]);
}

/* C' = J C J^T (+ Q when given) */
void orc_transport_cov(const double *J, const double *C, const double *Q, double *Cp)
{
    double JC[36], Jt[36];
    mat6_mul(J, C, JC);
    mat6_transpose(J, Jt);
    mat6_mul(JC, Jt, Cp);
    if (Q)
        for (int i = 0; i < 36; ++i) Cp[i] += Q[i];
}

/* chi2 increment of hit m against the prediction (xp, Cp):
 *   r = m - H xp,  S = H Cp H^T + V,  chi2 = r^T S^-1 r,   H = [I3 0]. */
double orc_chi2(const double *xp, const double *Cp, const double *m, const double *V)
{
    double S[9], Si[9], r[3];
    for (int i = 0; i < 3; ++i) {
        r[i] = m[i] - xp[i];
        for (int j = 0; j < 3; ++j) S[i * 3 + j] = Cp[i * 6 + j] + (i == j ? V[i] : 0.0);
    }
    mat3_inv(S, Si);
    double chi2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) chi2 += r[i] * Si[i * 3 + j] * r[j];
    return chi2;
}

/* Kalman update with hit m, measurement covariance V = diag(V[0..2]):
 *   K = Cp H^T S^-1,  x = xp + K r,
 *   C = (I - K H) Cp (I - K H)^T + K V K^T  (Joseph form), then symmetrised.
 * *dev gets max |C_joseph - C_standard| with C_standard = (I - K H) Cp. */
int orc_update(const double *xp, const double *Cp, const double *m, const double *V,
               double *x, double *C, double *chi2, double *dev)
{
    double S[9], Si[9], r[3], K[18];
    for (int i = 0; i < 3; ++i) {
        r[i] = m[i] - xp[i];
        for (int j = 0; j < 3; ++j) S[i * 3 + j] = Cp[i * 6 + j] + (i == j ? V[i] : 0.0);
    }
    mat3_inv(S, Si);
    double c2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c2 += r[i] * Si[i * 3 + j] * r[j];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += Cp[i * 6 + k] * Si[k * 3 + j];
            K[i * 3 + j] = acc;
        }
    for (int i = 0; i < 6; ++i) {
        double acc = 0.0;
        for (int j = 0; j < 3; ++j) acc += K[i * 3 + j] * r[j];
        x[i] = xp[i] + acc;
    }
    double A[36], At[36], T[36], Cj[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) A[i * 6 + j] = (i == j ? 1.0 : 0.0) - (j < 3 ? K[i * 3 + j] : 0.0);
    mat6_mul(A, Cp, T);
    mat6_transpose(A, At);
    mat6_mul(T, At, Cj);
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += K[i * 3 + k] * V[k] * K[j * 3 + k];
            Cj[i * 6 + j] += acc;
        }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) C[i * 6 + j] = 0.5 * (Cj[i * 6 + j] + Cj[j * 6 + i]);
    if (dev) {
        double m_ = 0.0;
        for (int i = 0; i < 36; ++i) {
            double d = fabs(C[i] - T[i]);
            if (d > m_) m_ = d;
        }
        *dev = m_;
    }
    if (chi2) *chi2 = c2;
    return 0;
}

/* Positive-definiteness of the rank-5 covariance: Cholesky of P C P^T with
 * P mapping to (t . pos, z, px, py, pz), t = (-sin phi, cos phi, 0) the
 * transverse direction tangent to the cylinder at the current position.
 * Returns 1 when PD. */
int orc_pd5(const double *x, const double *C)
{
    double r = sqrt(x[0] * x[0] + x[1] * x[1]);
    double P[30];
    memset(P, 0, sizeof P);
    if (r > 0) {
        P[0 * 6 + 0] = -x[1] / r;
        P[0 * 6 + 1] = x[0] / r;
    } else {
        P[0 * 6 + 1] = 1.0;
    }
    P[1 * 6 + 2] = 1.0;
    P[2 * 6 + 3] = 1.0;
    P[3 * 6 + 4] = 1.0;
    P[4 * 6 + 5] = 1.0;
    double M[25];
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 6; ++k)
                for (int l = 0; l < 6; ++l) acc += P[i * 6 + k] * C[k * 6 + l] * P[j * 6 + l];
            M[i * 5 + j] = acc;
        }
    double Lc[25];
    memset(Lc, 0, sizeof Lc);
    for (int j = 0; j < 5; ++j) {
        double d = M[j * 5 + j];
        for (int k = 0; k < j; ++k) d -= Lc[j * 5 + k] * Lc[j * 5 + k];
        if (!(d > 0.0)) return 0;
        Lc[j * 5 + j] = sqrt(d);
        for (int i = j + 1; i < 5; ++i) {
            double v = M[i * 5 + j];
            for (int k = 0; k < j; ++k) v -= Lc[i * 5 + k] * Lc[j * 5 + k];
            Lc[i * 5 + j] = v / Lc[j * 5 + j];
        }
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Track fit (Sec. 2): with the hit set fixed, apply propagate + update layer
 * by layer, no branching.
 *   seed_par [n][6], seed_cov [n][36], a_coef [n] (= q C_LIGHT Bz),
 *   hits [L][n][3], valid [L][n] (0: no hit, propagate only),
 *   radius [L], V [3] diagonal measurement variances, x_x0 [L] layer
 *   thickness in radiation lengths (NULL: no material) and the particle mass
 *   of the scattering model.
 * Outputs: out_par [n][6], out_cov [n][36] (state after the last layer
 * processed), chi2 [L][n] (-1 where no update), status [n].               */
int orc_fit(int64_t n, int n_layers, const double *radius, const double *V,
            const double *seed_par, const double *seed_cov, const double *a_coef,
            const double *hits, const uint8_t *valid, double *out_par, double *out_cov,
            double *chi2, int32_t *status, const double *x_x0, double mass, int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t t = 0; t < n; ++t) {
        double x[6], C[36], xp[6], Cp[36], J[36];
        memcpy(x, seed_par + 6 * t, sizeof x);
        memcpy(C, seed_cov + 36 * t, sizeof C);
        int32_t stat = 0;
        int stopped = 0;
        for (int l = 0; l < n_layers; ++l) {
            double *c2 = chi2 + (int64_t)l * n + t;
            *c2 = -1.0;
            if (stopped) continue;
            int st = orc_propagate(x, a_coef[t], radius[l], xp, J, NULL);
            if (st) {
                stat |= st;
                stopped = 1;
                continue;
            }
            if (x_x0 && x_x0[l] > 0.0) {
                double Q[36];
                orc_scattering_q(xp, x_x0[l], mass, Q);
                orc_transport_cov(J, C, Q, Cp);
            } else {
                orc_transport_cov(J, C, NULL, Cp);
            }
            if (valid[(int64_t)l * n + t]) {
                const double *m = hits + ((int64_t)l * n + t) * 3;
                orc_update(xp, Cp, m, V, x, C, c2, NULL);
            } else {
                memcpy(x, xp, sizeof x);
                memcpy(C, Cp, sizeof C);
                stat |= ORC_NO_HIT;
            }
        }
        /* positive-definiteness of the final covariance */
        if (!orc_pd5(x, C)) stat |= ORC_NOT_PD;
        memcpy(out_par + 6 * t, x, sizeof x);
        memcpy(out_cov + 36 * t, C, sizeof C);
        status[t] = stat;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Combinatorial track building with the clone engine (Sec. 3): per layer,
 * every live candidate of a seed is propagated, the chi2 increment of every
 * hit of the layer is computed (all hits, no binning), every hit with
 * chi2 < cut becomes a child (parent, hit, chi2_tot, nHits); a candidate with
 * no such hit gives one "miss" child (propagated, not updated).  The children
 * of a seed are ranked by (nHits desc, chi2_tot asc, parent rank asc, hit id
 * asc) and only the first max_cands are materialised (copied and updated),
 * after the bookkeeping list is complete.  max_cands = 1 is the best-hit
 * approach. */

#define ORC_MAX_LAYERS 64

typedef struct {
    double x[6], C[36];
    double chi2;
    int nhits;
    int stopped;
    int32_t status;
    int32_t hit[ORC_MAX_LAYERS];
} orc_cand;

typedef struct {
    int parent;  /* rank of the parent candidate */
    int32_t hit; /* hit id within the layer, -1 = miss */
    double chi2_tot;
    int nhits;
} orc_child;

static int child_cmp(const void *pa, const void *pb)
{
    const orc_child *a = (const orc_child *)pa, *b = (const orc_child *)pb;
    if (a->nhits != b->nhits) return a->nhits > b->nhits ? -1 : 1;
    if (a->chi2_tot != b->chi2_tot) return a->chi2_tot < b->chi2_tot ? -1 : 1;
    if (a->parent != b->parent) return a->parent < b->parent ? -1 : 1;
    if (a->hit != b->hit) return a->hit < b->hit ? -1 : 1;
    return 0;
}

/* Inputs: n_seeds seeds (seed_par [n][6], seed_cov [n][36], a_coef [n],
 * seed_event [n]); n_layers build layers at radius[]; hits of (event e,
 * layer l) are hits[hit_off[e*n_layers + l] .. hit_off[e*n_layers + l + 1])
 * as [.][3]; the hit id is the index within that segment.
 * Outputs per seed s and candidate rank k < max_cands:
 *   cand_par [s][k][6], cand_cov [s][k][36], cand_chi2 [s][k], cand_nhits [s][k],
 *   cand_hits [s][k][n_layers] (hit id or -1), cand_status [s][k];
 *   n_cands [s].  Candidate 0 is the best (nHits desc, chi2_tot asc). */
int orc_build(int64_t n_seeds, int n_layers, const double *radius, const double *V,
              double chi2_cut, int max_cands, const double *seed_par, const double *seed_cov,
              const double *a_coef, const int32_t *seed_event, const double *hits,
              const int64_t *hit_off, double *cand_par, double *cand_cov, double *cand_chi2,
              int32_t *cand_nhits, int32_t *cand_hits, int32_t *cand_status, int32_t *n_cands,
              const double *x_x0, double mass, int n_threads)
{
    if (n_layers > ORC_MAX_LAYERS || max_cands < 1) return -1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t sd = 0; sd < n_seeds; ++sd) {
        orc_cand *cur = (orc_cand *)calloc((size_t)max_cands, sizeof(orc_cand));
        orc_cand *nxt = (orc_cand *)calloc((size_t)max_cands, sizeof(orc_cand));
        double *xps = (double *)malloc(sizeof(double) * 6 * (size_t)max_cands);
        double *Cps = (double *)malloc(sizeof(double) * 36 * (size_t)max_cands);
        int ncur = 1;
        memcpy(cur[0].x, seed_par + 6 * sd, sizeof cur[0].x);
        memcpy(cur[0].C, seed_cov + 36 * sd, sizeof cur[0].C);
        cur[0].chi2 = 0.0;
        cur[0].nhits = 0;
        for (int l = 0; l < n_layers; ++l) cur[0].hit[l] = -1;
        int e = seed_event[sd];
        for (int l = 0; l < n_layers; ++l) {
            int64_t h0 = hit_off[(int64_t)e * n_layers + l], h1 = hit_off[(int64_t)e * n_layers + l + 1];
            /* bookkeeping list of all compatible (parent, hit) pairs */
            size_t cap = 64, nch = 0;
            orc_child *ch = (orc_child *)malloc(cap * sizeof(orc_child));
            for (int c = 0; c < ncur; ++c) {
                orc_cand *pc = &cur[c];
                int found = 0;
                if (!pc->stopped) {
                    double J[36];
                    int st = orc_propagate(pc->x, a_coef[sd], radius[l], xps + 6 * c, J, NULL);
                    if (st) {
                        pc->stopped = 1;
                        pc->status |= st;
                    } else {
                        if (x_x0 && x_x0[l] > 0.0) {
                            double Q[36];
                            orc_scattering_q(xps + 6 * c, x_x0[l], mass, Q);
                            orc_transport_cov(J, pc->C, Q, Cps + 36 * c);
                        } else {
                            orc_transport_cov(J, pc->C, NULL, Cps + 36 * c);
                        }
                        for (int64_t h = h0; h < h1; ++h) {
                            double c2 = orc_chi2(xps + 6 * c, Cps + 36 * c, hits + 3 * h, V);
                            if (c2 < chi2_cut) {
                                if (nch == cap) {
                                    cap *= 2;
                                    ch = (orc_child *)realloc(ch, cap * sizeof(orc_child));
                                }
                                ch[nch].parent = c;
                                ch[nch].hit = (int32_t)(h - h0);
                                ch[nch].chi2_tot = pc->chi2 + c2;
                                ch[nch].nhits = pc->nhits + 1;
                                ++nch;
                                found = 1;
                            }
                        }
                    }
                }
                if (!found) {
                    if (nch == cap) {
                        cap *= 2;
                        ch = (orc_child *)realloc(ch, cap * sizeof(orc_child));
                    }
                    ch[nch].parent = c;
                    ch[nch].hit = -1;
                    ch[nch].chi2_tot = pc->chi2;
                    ch[nch].nhits = pc->nhits;
                    ++nch;
                }
            }
            qsort(ch, nch, sizeof(orc_child), child_cmp);
            int nkeep = (int)(nch < (size_t)max_cands ? nch : (size_t)max_cands);
            /* clone engine: copy and update only the kept children */
            for (int k = 0; k < nkeep; ++k) {
                orc_cand *pc = &cur[ch[k].parent];
                orc_cand *nc = &nxt[k];
                *nc = *pc;
                if (pc->stopped) continue;
                if (ch[k].hit >= 0) {
                    double c2;
                    orc_update(xps + 6 * ch[k].parent, Cps + 36 * ch[k].parent,
                               hits + 3 * (h0 + ch[k].hit), V, nc->x, nc->C, &c2, NULL);
                    nc->chi2 = pc->chi2 + c2;
                    nc->nhits = pc->nhits + 1;
                } else {
                    memcpy(nc->x, xps + 6 * ch[k].parent, sizeof nc->x);
                    memcpy(nc->C, Cps + 36 * ch[k].parent, sizeof nc->C);
                    nc->status |= ORC_NO_HIT;
                }
                nc->hit[l] = ch[k].hit;
            }
            free(ch);
            orc_cand *tmp = cur;
            cur = nxt;
            nxt = tmp;
            ncur = nkeep;
        }
        n_cands[sd] = ncur;
        for (int k = 0; k < max_cands; ++k) {
            int64_t o = sd * max_cands + k;
            if (k < ncur) {
                if (!orc_pd5(cur[k].x, cur[k].C)) cur[k].status |= ORC_NOT_PD;
                memcpy(cand_par + 6 * o, cur[k].x, sizeof cur[k].x);
                memcpy(cand_cov + 36 * o, cur[k].C, sizeof cur[k].C);
                cand_chi2[o] = cur[k].chi2;
                cand_nhits[o] = cur[k].nhits;
                cand_status[o] = cur[k].status;
                for (int l = 0; l < n_layers; ++l) cand_hits[o * n_layers + l] = cur[k].hit[l];
            } else {
                memset(cand_par + 6 * o, 0, 6 * sizeof(double));
                memset(cand_cov + 36 * o, 0, 36 * sizeof(double));
                cand_chi2[o] = 0.0;
                cand_nhits[o] = 0;
                cand_status[o] = 0;
                for (int l = 0; l < n_layers; ++l) cand_hits[o * n_layers + l] = -1;
            }
        }
        free(cur);
        free(nxt);
        free(xps);
        free(Cps);
    }
    return 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
