/*
 * bs_oracle.c -- plain, slow, FP64 CPU oracle for the Biot-Savart velocity on
 * tetrahedral meshes (Carley, "Evaluation of Biot-Savart integrals on
 * tetrahedral meshes").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes, for every evaluation point x, summing tets in ascending
 * order (one point per OpenMP iteration, each point's sum sequential so the
 * result does not depend on the thread count):
 *
 *   far tet  (|x - centroid|^2 > (far_ratio * circumradius)^2):
 *       tet Gauss rule applied to Eq. 1,
 *       v += -(1/4pi) sum_q w_q |V| (x - x_q) x omega(x_q) / |x - x_q|^3
 *   near tet (otherwise), for every direction (n, m) of Eq. 3:
 *       optional pre-check of Section 2.1 (rejects only lines that provably
 *       miss the tet), Moller-Trumbore on each of the 4 faces (Section 2.1),
 *       chord [R0, R1] = [min, max] of the hits, omega at each end by the face
 *       area coordinates, and the chord integral of Eq. 5 with the sign of R
 *       kept (a segment with R0 < 0 < R1 is split at R = 0):
 *       v += k_nm * s_nm x integral_{R0}^{R1} sign(R) omega dR,
 *       k_nm = (pi/16) sin(phi_n) w_n w_m,
 *       or (near_rule 1) the exact integral of Eq. 1 over the tet
 *       (orc_tet_analytic), the analytic near-field evaluation that
 *       Section 1 sets the ray rule against.
 *
 * Readings of the paper taken here (the printed formulas are at odds with
 * Eq. 1 in two places):
 *   - Eq. 2 needs a factor sign(R): with theta covering [0, pi] only, the
 *     half-line R < 0 stands for the opposite direction -s, whose integrand
 *     is (-s) x omega.
 *   - The prefactor of Eq. 3 is (1/4pi)(pi/2)^2 = pi/16, from mapping both
 *     angular ranges [0, pi] onto the Gauss interval [-1, 1].
 *   - The pre-check of Section 2.1 rejects a line when
 *     (r.s)^2 < |r|^2 - 2 h^2 (r = x -> vertex, h = longest edge); then the
 *     line passes farther than sqrt(2) h from a vertex while every point of
 *     the tet lies within h of it, so no minimum |r| is needed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_ORDER -2

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                     */
/* ------------------------------------------------------------------------ */
static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [-1, 1] (Eq. 3: nodes t_i, weights w_i)            */
/* Newton iteration on P_n from the three-term recurrence                   */
/* (k P_k = (2k-1) x P_{k-1} - (k-1) P_{k-2}), weights 2/((1-x^2) P_n'(x)^2). */
/* Output ascending in t.                                                   */
/* ------------------------------------------------------------------------ */
static void legendre_eval(int n, double x, double *pn, double *dpn)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) { *pn = 1.0; *dpn = 0.0; return; }
    for (int k = 2; k <= n; k++) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    /* P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1) */
    *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

int orc_gauss_legendre(int n, double *t, double *w)
{
    if (n < 1 || !t || !w) return ORC_ERR_ARG;
    for (int i = 0; i < n; i++) {
        /* i-th root counted from +1 downwards */
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        double pn, dpn;
        for (int it = 0; it < 100; it++) {
            legendre_eval(n, x, &pn, &dpn);
            double dx = pn / dpn;
            x -= dx;
            if (fabs(dx) <= 1e-16) break;
        }
        legendre_eval(n, x, &pn, &dpn);
        t[n - 1 - i] = x;
        w[n - 1 - i] = 2.0 / ((1.0 - x * x) * dpn * dpn);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Jacobi rule on [0, 1] for the weight (1-u)^alpha (alpha = 0,1,2),   */
/* used by the conical-product tet rules.  Nodes: roots of the Jacobi       */
/* polynomial P_k^(alpha,0)(2u-1), located by a sign-change scan and refined */
/* by bisection.  Weights: the interpolatory rule, i.e. the k x k moment    */
/* system sum_i w_i u_i^m = int_0^1 u^m (1-u)^alpha du, m = 0..k-1, solved  */
/* by Gaussian elimination with partial pivoting.                           */
/* ------------------------------------------------------------------------ */
static double jacobi_eval(int n, double a, double b, double x)
{
    /* standard three-term recurrence for P_n^(a,b) on [-1, 1] */
    if (n == 0) return 1.0;
    double p0 = 1.0;
    double p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
    for (int k = 2; k <= n; k++) {
        double s = 2.0 * k + a + b;
        double c1 = 2.0 * k * (k + a + b) * (s - 2.0);
        double c2 = (s - 1.0) * (s * (s - 2.0) * x + a * a - b * b);
        double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
        double p2 = (c2 * p1 - c3 * p0) / c1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

static double beta_moment(int m, int alpha)
{
    /* int_0^1 u^m (1-u)^alpha du = m! alpha! / (m + alpha + 1)! */
    double num = 1.0, den = 1.0;
    for (int i = 2; i <= m; i++) num *= i;
    for (int i = 2; i <= alpha; i++) num *= i;
    for (int i = 2; i <= m + alpha + 1; i++) den *= i;
    return num / den;
}

int orc_gauss_jacobi01(int k, int alpha, double *u, double *w)
{
    if (k < 1 || k > 16 || alpha < 0 || alpha > 4 || !u || !w) return ORC_ERR_ARG;
    /* roots in x on (-1, 1) */
    const int scan = 200000;
    int found = 0;
    double xa = -1.0, fa = jacobi_eval(k, alpha, 0.0, xa);
    for (int s = 1; s <= scan && found < k; s++) {
        double xb = -1.0 + 2.0 * s / scan;
        double fb = jacobi_eval(k, alpha, 0.0, xb);
        if (fa == 0.0) {
            u[found++] = 0.5 * (xa + 1.0);
        } else if (fa * fb < 0.0) {
            double lo = xa, hi = xb, flo = fa;
            for (int it = 0; it < 200; it++) {
                double mid = 0.5 * (lo + hi);
                double fm = jacobi_eval(k, alpha, 0.0, mid);
                if (fm == 0.0) { lo = hi = mid; break; }
                if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
                if (hi - lo <= 1e-17) break;
            }
            u[found++] = 0.5 * (0.5 * (lo + hi) + 1.0);
        }
        xa = xb;
        fa = fb;
    }
    if (found != k) return ORC_ERR_ARG;
    /* moment system A w = mu, A[m][i] = u_i^m */
    double A[16][17];
    for (int m = 0; m < k; m++) {
        for (int i = 0; i < k; i++) A[m][i] = pow(u[i], m);
        A[m][k] = beta_moment(m, alpha);
    }
    for (int c = 0; c < k; c++) {
        int piv = c;
        for (int r = c + 1; r < k; r++)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c)
            for (int j = 0; j <= k; j++) { double tmp = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = tmp; }
        for (int r = c + 1; r < k; r++) {
            double f = A[r][c] / A[c][c];
            for (int j = c; j <= k; j++) A[r][j] -= f * A[c][j];
        }
    }
    for (int r = k - 1; r >= 0; r--) {
        double s = A[r][k];
        for (int j = r + 1; j < k; j++) s -= A[r][j] * w[j];
        w[r] = s / A[r][r];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Tet quadrature rules for the far field (Section 1: Gaussian quadrature   */
/* for tets far from x).  Barycentric points bary[q][4] and weights w[q]    */
/* summing to 1 (fractions of |V|).                                          */
/*   order 1 : centroid (degree 1)                                           */
/*   order 4 : symmetric rule a = (5+3 sqrt5)/20, b = (5-sqrt5)/20 (degree 2)*/
/*   order k^3, k = 2,3,4 : conical product rule (degree 2k-1) over the     */
/*      collapsed map xi1 = u, xi2 = (1-u) v, xi3 = (1-u)(1-v) t with       */
/*      Gauss-Jacobi in u (alpha 2), v (alpha 1) and Gauss-Legendre in t.   */
/* ------------------------------------------------------------------------ */
int orc_tet_rule(int order, double *bary, double *w)
{
    if (!bary || !w) return ORC_ERR_ARG;
    if (order == 1) {
        for (int i = 0; i < 4; i++) bary[i] = 0.25;
        w[0] = 1.0;
        return ORC_OK;
    }
    if (order == 4) {
        double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0, b = (5.0 - sqrt(5.0)) / 20.0;
        for (int q = 0; q < 4; q++) {
            for (int i = 0; i < 4; i++) bary[4 * q + i] = (i == q) ? a : b;
            w[q] = 0.25;
        }
        return ORC_OK;
    }
    int k = 0;
    if (order == 8) k = 2;
    else if (order == 27) k = 3;
    else if (order == 64) k = 4;
    else return ORC_ERR_ORDER;
    double uu[16], wu[16], vv[16], wv[16], tt[16], wt[16];
    if (orc_gauss_jacobi01(k, 2, uu, wu) || orc_gauss_jacobi01(k, 1, vv, wv) || orc_gauss_jacobi01(k, 0, tt, wt))
        return ORC_ERR_ARG;
    int q = 0;
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++)
            for (int l = 0; l < k; l++) {
                double x1 = uu[i];
                double x2 = (1.0 - uu[i]) * vv[j];
                double x3 = (1.0 - uu[i]) * (1.0 - vv[j]) * tt[l];
                bary[4 * q + 0] = 1.0 - x1 - x2 - x3;
                bary[4 * q + 1] = x1;
                bary[4 * q + 2] = x2;
                bary[4 * q + 3] = x3;
                /* reference tet volume is 1/6; weights as fractions of |V| */
                w[q] = 6.0 * wu[i] * wv[j] * wt[l];
                q++;
            }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Direction table of Eq. 3 / Section 2.2 step 3.                            */
/* Line index l = n * n_theta + m, n over phi (N = n_phi points),           */
/* m over theta (M = n_theta points).                                       */
/* ------------------------------------------------------------------------ */
int orc_directions(int n_phi, int n_theta, double *s, double *k)
{
    if (n_phi < 1 || n_theta < 1 || n_phi > 512 || n_theta > 512 || !s || !k) return ORC_ERR_ARG;
    double tN[512], wN[512], tM[512], wM[512];
    orc_gauss_legendre(n_phi, tN, wN);
    orc_gauss_legendre(n_theta, tM, wM);
    for (int n = 0; n < n_phi; n++) {
        double phi = (1.0 + tN[n]) * M_PI / 2.0;
        for (int m = 0; m < n_theta; m++) {
            double theta = (1.0 + tM[m]) * M_PI / 2.0;
            int l = n * n_theta + m;
            s[3 * l + 0] = sin(phi) * cos(theta);
            s[3 * l + 1] = sin(phi) * sin(theta);
            s[3 * l + 2] = cos(phi);
            k[l] = (M_PI / 16.0) * sin(phi) * wN[n] * wM[m];
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Moller-Trumbore ray/triangle test (Section 2.1), two-sided, for the full  */
/* line o + t d, t in (-inf, inf).  Returns 1 on a hit with (t, u, v);       */
/* the hit point is (1-u-v) p0 + u p1 + v p2.                                */
/* eps_det: |det| <= eps_det |e1||e2| counts as parallel (no hit).           */
/* eps_b  : area coordinates accepted in [-eps_b, 1+eps_b].                  */
/* ------------------------------------------------------------------------ */
int orc_moller_trumbore(const double *o, const double *d, const double *p0, const double *p1, const double *p2,
                        double eps_det, double eps_b, double *t, double *u, double *v)
{
    double e1[3], e2[3], P[3], T[3], Q[3];
    sub3(p1, p0, e1);
    sub3(p2, p0, e2);
    cross3(d, e2, P);
    double det = dot3(e1, P);
    if (fabs(det) <= eps_det * sqrt(dot3(e1, e1) * dot3(e2, e2))) return 0;
    double inv = 1.0 / det;
    sub3(o, p0, T);
    double uu = dot3(T, P) * inv;
    if (uu < -eps_b || uu > 1.0 + eps_b) return 0;
    cross3(T, e1, Q);
    double vv = dot3(d, Q) * inv;
    if (vv < -eps_b || uu + vv > 1.0 + eps_b) return 0;
    *t = dot3(e2, Q) * inv;
    *u = uu;
    *v = vv;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Per-tet geometry: centroid, circumradius, longest edge.                   */
/* Circumcentre p solves 2 (v_i - v_0) . p = |v_i|^2 - |v_0|^2, i = 1..3     */
/* (Cramer's rule), circumradius = |p - v_0|.                               */
/* ------------------------------------------------------------------------ */
static double det3(const double *a, const double *b, const double *c)
{
    double bc[3];
    cross3(b, c, bc);
    return dot3(a, bc);
}

int orc_tet_geometry(const double *v /*[4][3]*/, double *centroid, double *circumradius, double *hmax, double *volume)
{
    for (int j = 0; j < 3; j++) centroid[j] = 0.25 * (v[0 + j] + v[3 + j] + v[6 + j] + v[9 + j]);
    double r1[3], r2[3], r3[3], rhs[3];
    for (int j = 0; j < 3; j++) {
        r1[j] = 2.0 * (v[3 + j] - v[j]);
        r2[j] = 2.0 * (v[6 + j] - v[j]);
        r3[j] = 2.0 * (v[9 + j] - v[j]);
    }
    rhs[0] = dot3(v + 3, v + 3) - dot3(v, v);
    rhs[1] = dot3(v + 6, v + 6) - dot3(v, v);
    rhs[2] = dot3(v + 9, v + 9) - dot3(v, v);
    /* rows r1, r2, r3; solve by Cramer using columns */
    double c0[3] = {r1[0], r2[0], r3[0]}, c1[3] = {r1[1], r2[1], r3[1]}, c2[3] = {r1[2], r2[2], r3[2]};
    double D = det3(c0, c1, c2);
    double p[3];
    p[0] = det3(rhs, c1, c2) / D;
    p[1] = det3(c0, rhs, c2) / D;
    p[2] = det3(c0, c1, rhs) / D;
    double dp[3];
    sub3(p, v, dp);
    *circumradius = sqrt(dot3(dp, dp));
    double h2 = 0.0;
    for (int a = 0; a < 4; a++)
        for (int b = a + 1; b < 4; b++) {
            double e[3];
            sub3(v + 3 * b, v + 3 * a, e);
            double l2 = dot3(e, e);
            if (l2 > h2) h2 = l2;
        }
    *hmax = sqrt(h2);
    double e1[3], e2[3], e3[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    sub3(v + 9, v, e3);
    *volume = fabs(det3(e1, e2, e3)) / 6.0;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* One line through x with direction s against one tet (Section 2.1):        */
/* pre-check (optional), Moller-Trumbore on the 4 faces, chord ends and the  */
/* signed chord integral J = int_{R0}^{R1} sign(R) omega dR (Eq. 5 with the  */
/* sign of R kept).  Returns 1 when the chord is longer than tau * h and     */
/* contributes, 0 otherwise.  Outputs R0, R1 and J.                          */
/* Face f is the face opposite vertex f.                                     */
/* ------------------------------------------------------------------------ */
static const int FACE_VERTS[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};

int orc_line_tet(const double *x, const double *s, const double *v /*[4][3]*/, const double *om /*[4][3]*/,
                 double hmax, int use_precheck, double eps_b, double tau, double *R0out, double *R1out, double *J)
{
    J[0] = J[1] = J[2] = 0.0;
    *R0out = *R1out = 0.0;
    if (use_precheck) {
        /* Section 2.1: r = x -> vertex 0, reject if (r.s)^2 < |r|^2 - 2 h^2 */
        double r[3];
        sub3(v, x, r);
        double rs = dot3(r, s);
        if (rs * rs < dot3(r, r) - 2.0 * hmax * hmax) return 0;
    }
    int nh = 0;
    double R0 = 0.0, R1 = 0.0, w0[3] = {0, 0, 0}, w1[3] = {0, 0, 0};
    for (int f = 0; f < 4; f++) {
        int a = FACE_VERTS[f][0], b = FACE_VERTS[f][1], c = FACE_VERTS[f][2];
        double t, u, vv;
        if (!orc_moller_trumbore(x, s, v + 3 * a, v + 3 * b, v + 3 * c, 1e-12, eps_b, &t, &u, &vv)) continue;
        double w[3];
        for (int j = 0; j < 3; j++) w[j] = (1.0 - u - vv) * om[3 * a + j] + u * om[3 * b + j] + vv * om[3 * c + j];
        if (nh == 0) {
            R0 = R1 = t;
            memcpy(w0, w, sizeof w);
            memcpy(w1, w, sizeof w);
        } else {
            if (t < R0) { R0 = t; memcpy(w0, w, sizeof w); }
            if (t > R1) { R1 = t; memcpy(w1, w, sizeof w); }
        }
        nh++;
    }
    if (nh < 2 || !(R1 - R0 > tau * hmax)) return 0;
    *R0out = R0;
    *R1out = R1;
    if (R0 >= 0.0) {
        for (int j = 0; j < 3; j++) J[j] = 0.5 * (R1 - R0) * (w0[j] + w1[j]);
    } else if (R1 <= 0.0) {
        for (int j = 0; j < 3; j++) J[j] = -0.5 * (R1 - R0) * (w0[j] + w1[j]);
    } else {
        /* split at R = 0; omega there by linear interpolation along the chord */
        double f = (0.0 - R0) / (R1 - R0);
        for (int j = 0; j < 3; j++) {
            double wx = w0[j] + f * (w1[j] - w0[j]);
            J[j] = 0.5 * R1 * (wx + w1[j]) - 0.5 * (0.0 - R0) * (w0[j] + wx);
        }
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Exact Eq. 1 over one tet with linear vorticity: the analytic near-field   */
/* evaluation of Section 1 (the Stokes-theorem reduction of the volume       */
/* integral to face integrals and then to closed-form edge integrals, the    */
/* approach the paper compares its ray rule against).  Written out from the  */
/* calculus, with R = x - y, rho = |R|:                                      */
/*   R x omega / rho^3 = grad_y(1/rho) x omega                               */
/*                     = curl_y(omega / rho) - (curl omega) / rho,           */
/* and by the divergence theorem (n outward, curl omega constant on T)      */
/*   v = -(1/4pi) [ sum_f n_f x int_f omega/rho dS                           */
/*                  - (curl omega) int_T 1/rho dV ],                        */
/*   int_T 1/rho dV = (1/2) sum_f h_f int_f 1/rho dS,  h_f = n_f.(y - x)    */
/* (div_y((y - x)/rho) = 2/rho).  With omega(y) = omega(x) + G (y - x),     */
/* G = grad omega, and p = x + h n the foot of x on the face plane:         */
/*   int_f omega/rho = omega(x) I0 + G (Ip + h n I0),                       */
/*   I0 = int_f 1/rho dS,  Ip = int_f (y - p)/rho dS.                       */
/* In the plane, Ip = int grad_s(rho) = sum_edges m_e int_e rho dl and      */
/* 1/rho = div_s((y - p)(rho - |h|)/|y - p|^2), so per edge (unit tangent t, */
/* in-plane outward normal m, l = (y - x).t along it, P0 = (y - x).m,       */
/* R0^2 = P0^2 + h^2, R at the ends, f = int dl / rho):                     */
/*   Ip += m (R0^2 f + l+ R+ - l- R-) / 2,                                  */
/*   I0 += P0 f - |h| [atan(P0 l/(R0^2 + |h| R))]_{l-}^{l+}.                 */
/* That is one logarithm and two arc tangents per face edge: 12 and 24 per   */
/* tet, the count the paper quotes for the analytic formulae.  f is taken in */
/* the form free of cancellation for the signs of l-, l+.  When x is on an   */
/* edge's line (R0 = 0) that edge's terms vanish (P0 f, R0^2 f -> 0); when   */
/* P0 = 0 the arc tangent term vanishes.                                     */
/*   v, om [4][3]; vel [3] overwritten.                                       */
/* ------------------------------------------------------------------------ */
static void orc_face_integrals(const double *x, const double *ya, const double *yb, const double *yc,
                               const double *n, double *h_out, double *I0_out, double *Ip)
{
    double d[3];
    sub3(ya, x, d);
    const double h = dot3(n, d), ah = fabs(h);
    const double *ends[3][2] = {{ya, yb}, {yb, yc}, {yc, ya}};
    double I0 = 0.0;
    Ip[0] = Ip[1] = Ip[2] = 0.0;
    for (int e = 0; e < 3; e++) {
        const double *u = ends[e][0], *w = ends[e][1];
        double t[3], m[3], um[3], wm[3];
        sub3(w, u, t);
        const double L = sqrt(dot3(t, t));
        for (int j = 0; j < 3; j++) t[j] /= L;
        cross3(t, n, m);
        sub3(u, x, um);
        sub3(w, x, wm);
        const double lm = dot3(um, t), lp = dot3(wm, t);
        const double P0 = dot3(um, m);
        const double Rm = sqrt(dot3(um, um)), Rp = sqrt(dot3(wm, wm));
        const double R02 = P0 * P0 + h * h;
        double f = 0.0;
        if (R02 > 1e-26 * L * L) {
            if (lm >= 0.0)
                f = log((Rp + lp) / (Rm + lm));
            else if (lp <= 0.0)
                f = log((Rm - lm) / (Rp - lp));
            else
                f = log((Rp + lp) * (Rm - lm) / R02);
        }
        double beta = 0.0;
        if (fabs(P0) > 1e-13 * L) beta = atan(P0 * lp / (R02 + ah * Rp)) - atan(P0 * lm / (R02 + ah * Rm));
        I0 += P0 * f - ah * beta;
        const double c = 0.5 * (R02 * f + lp * Rp - lm * Rm);
        for (int j = 0; j < 3; j++) Ip[j] += c * m[j];
    }
    *h_out = h;
    *I0_out = I0;
}

int orc_tet_analytic(const double *x, const double *v /*[4][3]*/, const double *om /*[4][3]*/, double *vel)
{
    /* barycentric gradients g_i (lambda_i(y) = g_i . (y - v_0) for i = 1..3) */
    double e1[3], e2[3], e3[3], n1[3], n2[3], n3[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    sub3(v + 9, v, e3);
    cross3(e2, e3, n1);
    cross3(e3, e1, n2);
    cross3(e1, e2, n3);
    const double V6 = dot3(e1, n1);
    if (V6 == 0.0) return ORC_ERR_ARG;
    const double *nn[3] = {n1, n2, n3};
    /* G[a][b] = d omega_a / d y_b = sum_i (omega_i - omega_0)_a g_i,b */
    double G[3][3] = {{0}};
    for (int i = 1; i <= 3; i++)
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) G[a][b] += (om[3 * i + a] - om[a]) * nn[i - 1][b] / V6;
    const double curl[3] = {G[2][1] - G[1][2], G[0][2] - G[2][0], G[1][0] - G[0][1]};
    double xm[3], wx[3];
    sub3(x, v, xm);
    for (int a = 0; a < 3; a++) wx[a] = om[a] + G[a][0] * xm[0] + G[a][1] * xm[1] + G[a][2] * xm[2];
    double S[3] = {0.0, 0.0, 0.0}, volint = 0.0;
    for (int f = 0; f < 4; f++) {
        const double *ya = v + 3 * FACE_VERTS[f][0], *yb = v + 3 * FACE_VERTS[f][1], *yc = v + 3 * FACE_VERTS[f][2];
        double ab[3], ac[3], n[3], od[3];
        sub3(yb, ya, ab);
        sub3(yc, ya, ac);
        cross3(ab, ac, n);
        const double nl = sqrt(dot3(n, n));
        for (int j = 0; j < 3; j++) n[j] /= nl;
        sub3(v + 3 * f, ya, od); /* vertex f is the one off face f */
        const double *p0 = ya, *p1 = yb, *p2 = yc;
        if (dot3(n, od) > 0.0) { /* point n outward and keep (p0, p1, p2) counter-clockwise about it */
            for (int j = 0; j < 3; j++) n[j] = -n[j];
            p1 = yc;
            p2 = yb;
        }
        double h, I0, Ip[3];
        orc_face_integrals(x, p0, p1, p2, n, &h, &I0, Ip);
        double q[3], Iw[3], nxI[3];
        for (int j = 0; j < 3; j++) q[j] = Ip[j] + h * n[j] * I0;
        for (int a = 0; a < 3; a++) Iw[a] = wx[a] * I0 + G[a][0] * q[0] + G[a][1] * q[1] + G[a][2] * q[2];
        cross3(n, Iw, nxI);
        for (int j = 0; j < 3; j++) S[j] += nxI[j];
        volint += 0.5 * h * I0;
    }
    const double c = -1.0 / (4.0 * M_PI);
    for (int j = 0; j < 3; j++) vel[j] = c * (S[j] - curl[j] * volint);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Velocity at points (the whole method).                                   */
/*   nodes [n_nodes][3], tets [n_tets][4] (int32), omega [n_nodes][3],       */
/*   pts [n_pts][3]; far_ratio >= 0 (INFINITY = every tet near);            */
/*   tet_order in {1, 4, 8, 27, 64}; n_theta, n_phi >= 1; near_rule 0: the  */
/*   ray rule of Section 2 for near tets, 1: the exact integral              */
/*   (orc_tet_analytic).  vel [n_pts][3] overwritten.  counts [n_pts][3]     */
/*   (near, far, ray hits; no hits under near_rule 1) or NULL.               */
/* ------------------------------------------------------------------------ */
int orc_velocity(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets, const double *omega,
                 const double *pts, int64_t n_pts, double far_ratio, int tet_order, int n_theta, int n_phi,
                 int use_precheck, double eps_b, double tau, int near_rule, double *vel, int32_t *counts)
{
    if (near_rule != 0 && near_rule != 1) return ORC_ERR_ARG;
    if (!nodes || !tets || !omega || !pts || !vel || n_pts < 0 || n_tets < 0 || n_nodes < 0) return ORC_ERR_ARG;
    if (n_theta < 1 || n_phi < 1 || n_theta > 512 || n_phi > 512) return ORC_ERR_ARG;
    double bary[64 * 4], wq[64];
    if (orc_tet_rule(tet_order, bary, wq)) return ORC_ERR_ORDER;
    const int nq = tet_order;
    const int L = n_theta * n_phi;
    double *S = (double *)malloc(sizeof(double) * 3 * L);
    double *K = (double *)malloc(sizeof(double) * L);
    /* per-tet geometry, computed once */
    double *cen = (double *)malloc(sizeof(double) * 3 * (n_tets > 0 ? n_tets : 1));
    double *rho = (double *)malloc(sizeof(double) * (n_tets > 0 ? n_tets : 1));
    double *hmx = (double *)malloc(sizeof(double) * (n_tets > 0 ? n_tets : 1));
    double *vol = (double *)malloc(sizeof(double) * (n_tets > 0 ? n_tets : 1));
    if (!S || !K || !cen || !rho || !hmx || !vol) {
        free(S); free(K); free(cen); free(rho); free(hmx); free(vol);
        return ORC_ERR_ARG;
    }
    orc_directions(n_phi, n_theta, S, K);
    for (int64_t e = 0; e < n_tets; e++) {
        double v[12];
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 3; j++) v[3 * i + j] = nodes[3 * (int64_t)tets[4 * e + i] + j];
        orc_tet_geometry(v, cen + 3 * e, rho + e, hmx + e, vol + e);
    }
    const double inv4pi = 1.0 / (4.0 * M_PI);

#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < n_pts; p++) {
        const double *x = pts + 3 * p;
        double acc[3] = {0.0, 0.0, 0.0};
        int32_t n_near = 0, n_far = 0, n_hit = 0;
        for (int64_t e = 0; e < n_tets; e++) {
            double v[12], om[12];
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 3; j++) {
                    v[3 * i + j] = nodes[3 * (int64_t)tets[4 * e + i] + j];
                    om[3 * i + j] = omega[3 * (int64_t)tets[4 * e + i] + j];
                }
            double dc[3];
            sub3(x, cen + 3 * e, dc);
            double thr = far_ratio * rho[e];
            int far = isinf(far_ratio) ? 0 : (dot3(dc, dc) > thr * thr);
            if (far) {
                n_far++;
                for (int q = 0; q < nq; q++) {
                    double xq[3] = {0, 0, 0}, wqv[3] = {0, 0, 0};
                    for (int i = 0; i < 4; i++)
                        for (int j = 0; j < 3; j++) {
                            xq[j] += bary[4 * q + i] * v[3 * i + j];
                            wqv[j] += bary[4 * q + i] * om[3 * i + j];
                        }
                    double r[3], rxw[3];
                    sub3(x, xq, r);
                    double R = sqrt(dot3(r, r));
                    cross3(r, wqv, rxw);
                    double f = -inv4pi * wq[q] * vol[e] / (R * R * R);
                    for (int j = 0; j < 3; j++) acc[j] += f * rxw[j];
                }
            } else if (near_rule == 1) {
                n_near++;
                double va[3];
                orc_tet_analytic(x, v, om, va);
                for (int j = 0; j < 3; j++) acc[j] += va[j];
            } else {
                n_near++;
                for (int l = 0; l < L; l++) {
                    double R0, R1, J[3];
                    if (!orc_line_tet(x, S + 3 * l, v, om, hmx[e], use_precheck, eps_b, tau, &R0, &R1, J)) continue;
                    n_hit++;
                    double sxJ[3];
                    cross3(S + 3 * l, J, sxJ);
                    for (int j = 0; j < 3; j++) acc[j] += K[l] * sxJ[j];
                }
            }
        }
        for (int j = 0; j < 3; j++) vel[3 * p + j] = acc[j];
        if (counts) {
            counts[3 * p + 0] = n_near;
            counts[3 * p + 1] = n_far;
            counts[3 * p + 2] = n_hit;
        }
    }
    free(S); free(K); free(cen); free(rho); free(hmx); free(vol);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Derivative of the all-ray velocity (every tet by the ray rule) at points  */
/* x along directions e.  The paper gives no vorticity update; the stretching */
/* term (omega . grad) v of the Lagrangian method is this derivative with     */
/* e = omega(x).  Along one line the rule integrates                          */
/*   J(x) = int sign(R) omega_h(x + R s) dR                                   */
/* (omega_h: the piecewise-linear vorticity, zero outside the mesh), so       */
/*   dJ/de = int sign(R) (e . grad omega_h) dR                                */
/*           + [sign(R) omega_h(R) dR/de] at the mesh boundary crossings,    */
/* the second term from the jump of omega_h to zero where the line leaves    */
/* the mesh (inside, omega_h is continuous and the chord ends of neighbouring */
/* tets cancel).  Per tet the first term is (|R1| - |R0|) (e . grad omega_T); */
/* for a chord end on a boundary face with normal n, dR/de = -(n . e)/(n . s) */
/* (moving x by e moves the line's crossing of the face plane), entering with */
/* the sign - at R0 and + at R1; sign(R) = 0 for |R| <= 1e-12 h (the point    */
/* itself).  dv/de = sum over lines k s x dJ/de.                              */
/*   pts, dirs [n_pts][3]; vel, dvel [n_pts][3] overwritten (vel: as          */
/*   orc_velocity with far_ratio = INFINITY).                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t a, b, c;
    int64_t slot; /* 4 * tet + face */
} orc_face;

static int face_cmp(const void *x, const void *y)
{
    const orc_face *p = (const orc_face *)x, *q = (const orc_face *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    if (p->c != q->c) return p->c < q->c ? -1 : 1;
    return p->slot < q->slot ? -1 : (p->slot > q->slot);
}

static void sort3i(int32_t *v)
{
    int32_t t;
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
    if (v[1] > v[2]) { t = v[1]; v[1] = v[2]; v[2] = t; }
    if (v[0] > v[1]) { t = v[0]; v[0] = v[1]; v[1] = t; }
}

int orc_velocity_dderiv(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                        const double *omega, const double *pts, const double *dirs, int64_t n_pts, int n_theta,
                        int n_phi, double eps_b, double tau, double *vel, double *dvel)
{
    if (!nodes || !tets || !omega || !pts || !dirs || !vel || !dvel || n_pts < 0 || n_tets < 0 || n_nodes < 0)
        return ORC_ERR_ARG;
    if (n_theta < 1 || n_phi < 1 || n_theta > 512 || n_phi > 512) return ORC_ERR_ARG;
    int rc = orc_velocity(nodes, n_nodes, tets, n_tets, omega, pts, n_pts, INFINITY, 1, n_theta, n_phi, 0, eps_b,
                          tau, 0, vel, NULL);
    if (rc) return rc;
    const int L = n_theta * n_phi;
    double *S = (double *)malloc(sizeof(double) * 3 * L);
    double *K = (double *)malloc(sizeof(double) * L);
    char *bnd = (char *)calloc((size_t)(n_tets > 0 ? 4 * n_tets : 1), 1); /* face on the mesh boundary */
    orc_face *F = (orc_face *)malloc(sizeof(orc_face) * (size_t)(n_tets > 0 ? 4 * n_tets : 1));
    if (!S || !K || !bnd || !F) {
        free(S); free(K); free(bnd); free(F);
        return ORC_ERR_ARG;
    }
    orc_directions(n_phi, n_theta, S, K);
    /* boundary faces: faces that belong to one tet only */
    for (int64_t e = 0; e < n_tets; e++)
        for (int f = 0; f < 4; f++) {
            int32_t v[3] = {tets[4 * e + FACE_VERTS[f][0]], tets[4 * e + FACE_VERTS[f][1]], tets[4 * e + FACE_VERTS[f][2]]};
            sort3i(v);
            F[4 * e + f].a = v[0];
            F[4 * e + f].b = v[1];
            F[4 * e + f].c = v[2];
            F[4 * e + f].slot = 4 * e + f;
        }
    qsort(F, (size_t)(4 * n_tets), sizeof(orc_face), face_cmp);
    for (int64_t i = 0; i < 4 * n_tets;) {
        int64_t j = i + 1;
        while (j < 4 * n_tets && F[j].a == F[i].a && F[j].b == F[i].b && F[j].c == F[i].c) j++;
        if (j - i == 1) bnd[F[i].slot] = 1;
        i = j;
    }
    free(F);

#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < n_pts; p++) {
        const double *x = pts + 3 * p, *ed = dirs + 3 * p;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t e = 0; e < n_tets; e++) {
            double v[12], om[12];
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 3; j++) {
                    v[3 * i + j] = nodes[3 * (int64_t)tets[4 * e + i] + j];
                    om[3 * i + j] = omega[3 * (int64_t)tets[4 * e + i] + j];
                }
            /* barycentric gradients (face planes) and e . grad omega_T */
            double e1[3], e2[3], e3[3], gl[4][3], c23[3], c31[3], c12[3];
            sub3(v + 3, v, e1);
            sub3(v + 6, v, e2);
            sub3(v + 9, v, e3);
            cross3(e2, e3, c23);
            cross3(e3, e1, c31);
            cross3(e1, e2, c12);
            double V6 = dot3(e1, c23);
            for (int j = 0; j < 3; j++) {
                gl[1][j] = c23[j] / V6;
                gl[2][j] = c31[j] / V6;
                gl[3][j] = c12[j] / V6;
                gl[0][j] = -(gl[1][j] + gl[2][j] + gl[3][j]);
            }
            double gw[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < 4; i++) {
                double ge = dot3(gl[i], ed);
                for (int j = 0; j < 3; j++) gw[j] += om[3 * i + j] * ge;
            }
            double hmax2 = 0.0;
            for (int a = 0; a < 4; a++)
                for (int b = a + 1; b < 4; b++) {
                    double d[3];
                    sub3(v + 3 * b, v + 3 * a, d);
                    if (dot3(d, d) > hmax2) hmax2 = dot3(d, d);
                }
            const double hmax = sqrt(hmax2);
            for (int l = 0; l < L; l++) {
                const double *s = S + 3 * l;
                int nh = 0, f0 = -1, f1 = -1;
                double R0 = 0.0, R1 = 0.0, w0[3] = {0, 0, 0}, w1[3] = {0, 0, 0};
                for (int f = 0; f < 4; f++) {
                    int a = FACE_VERTS[f][0], b = FACE_VERTS[f][1], c = FACE_VERTS[f][2];
                    double t, u, vv;
                    if (!orc_moller_trumbore(x, s, v + 3 * a, v + 3 * b, v + 3 * c, 1e-12, eps_b, &t, &u, &vv)) continue;
                    double w[3]; /* omega at the hit from the face's area coordinates */
                    for (int j = 0; j < 3; j++)
                        w[j] = om[3 * a + j] + u * (om[3 * b + j] - om[3 * a + j]) + vv * (om[3 * c + j] - om[3 * a + j]);
                    if (nh == 0 || t < R0) { R0 = t; f0 = f; memcpy(w0, w, sizeof w); }
                    if (nh == 0 || t > R1) { R1 = t; f1 = f; memcpy(w1, w, sizeof w); }
                    nh++;
                }
                if (nh < 2 || !(R1 - R0 > 0.0)) continue;
                double dJ[3];
                for (int j = 0; j < 3; j++) dJ[j] = (fabs(R1) - fabs(R0)) * gw[j];
                const int ends[2] = {f0, f1};
                const double Rs[2] = {R0, R1}, sgn_end[2] = {-1.0, 1.0};
                const double *ws[2] = {w0, w1};
                for (int k = 0; k < 2; k++) {
                    if (!bnd[4 * e + ends[k]]) continue;
                    const double R = Rs[k];
                    const double sg = fabs(R) <= 1e-12 * hmax ? 0.0 : (R > 0.0 ? 1.0 : -1.0);
                    if (sg == 0.0) continue;
                    /* normal of the end's face plane and dR/de = -(n . e)/(n . s) */
                    int a = FACE_VERTS[ends[k]][0], b = FACE_VERTS[ends[k]][1], c = FACE_VERTS[ends[k]][2];
                    double ea[3], eb[3], n[3];
                    sub3(v + 3 * b, v + 3 * a, ea);
                    sub3(v + 3 * c, v + 3 * a, eb);
                    cross3(ea, eb, n);
                    const double dR = -dot3(n, ed) / dot3(n, s);
                    for (int j = 0; j < 3; j++) dJ[j] += sgn_end[k] * sg * ws[k][j] * dR;
                }
                double sxd[3];
                cross3(s, dJ, sxd);
                for (int j = 0; j < 3; j++) acc[j] += K[l] * sxd[j];
            }
        }
        for (int j = 0; j < 3; j++) dvel[3 * p + j] = acc[j];
    }
    free(S); free(K); free(bnd);
    return ORC_OK;
}

/* Threads of the later OpenMP loops (n >= 1); no effect without OpenMP.  Results do not depend on it. */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
