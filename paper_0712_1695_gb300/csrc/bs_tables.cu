// bs_tables.cu -- quadrature tables computed on the device in float64.
//
//  * Gauss-Legendre nodes/weights and the direction table of Eq. 3
//    (Section 2.2 steps 2-3): phi_n = (1 + t_n) pi/2, theta_m = (1 + t_m) pi/2,
//    s_nm = (sin phi cos theta, sin phi sin theta, cos phi),
//    k_nm = (pi/16) sin(phi_n) w_n w_m  (the printed 1/(16 pi^2) does not follow
//    from Eq. 2; mapping both [0, pi] ranges to [-1, 1] gives (1/4pi)(pi/2)^2).
//  * Tet rules for the far field (Section 1): centroid, the symmetric 4-point
//    degree-2 rule, and conical-product rules with k^3 points (degree 2k-1)
//    from Gauss-Jacobi rules in the collapsed coordinates
//    xi1 = u, xi2 = (1-u) v, xi3 = (1-u)(1-v) t (Jacobian (1-u)^2 (1-v)).
//
// Roots by Newton iteration with deflation on the Jacobi polynomial
// P_n^(a,0) (a = 0 is Legendre); weights by the Gauss-Jacobi formula
// w = 2^(a+1) / ((1 - x^2) P_n'(x)^2) on [-1, 1] (weight (1-x)^a), mapped to
// [0, 1] with weight (1-u)^a by dividing by 2^(a+1).
#include <math.h>

#include "bs_internal.cuh"

namespace bs {
namespace {

__device__ double jacobi_p(int n, double a, double b, double x)
{
    if (n == 0) return 1.0;
    double p0 = 1.0, p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
    for (int k = 2; k <= n; ++k) {
        const double s = 2.0 * k + a + b;
        const double c1 = 2.0 * k * (k + a + b) * (s - 2.0);
        const double c2 = (s - 1.0) * (s * (s - 2.0) * x + a * a - b * b);
        const double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
        const double p2 = (c2 * p1 - c3 * p0) / c1;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// d/dx P_n^(a,0) = (n + a + 1)/2 * P_{n-1}^(a+1,1)
__device__ double jacobi_dp(int n, double a, double x)
{
    return n == 0 ? 0.0 : 0.5 * (n + a + 1.0) * jacobi_p(n - 1, a + 1.0, 1.0, x);
}

// All n roots of P_n^(a,0), descending, by deflated Newton.  One thread.
__device__ void jacobi_roots(int n, double a, double *x)
{
    for (int i = 0; i < n; ++i) {
        double r = cos(kPi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            const double f = jacobi_p(n, a, 0.0, r);
            const double df = jacobi_dp(n, a, r);
            double s = 0.0;
            for (int j = 0; j < i; ++j) s += 1.0 / (r - x[j]);
            const double dx = f / (df - f * s);
            r -= dx;
            if (fabs(dx) <= 1e-16) break;
        }
        x[i] = r;
    }
}

// Legendre roots are independent: one thread per root, Newton from the
// classical cosine guess (no deflation needed for P_n up to 256).
__device__ void legendre_root(int n, int i, double *t, double *w)
{
    double r = cos(kPi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
        const double f = jacobi_p(n, 0.0, 0.0, r);
        const double dx = f / jacobi_dp(n, 0.0, r);
        r -= dx;
        if (fabs(dx) <= 1e-16) break;
    }
    const double d = jacobi_dp(n, 0.0, r);
    t[n - 1 - i] = r;  // ascending
    w[n - 1 - i] = 2.0 / ((1.0 - r * r) * d * d);
}

__global__ void lines_kernel(int n_phi, int n_theta, float4 *f32, dbl4 *f64)
{
    __shared__ double tN[256], wN[256], tM[256], wM[256];
    for (int i = threadIdx.x; i < n_phi; i += blockDim.x) legendre_root(n_phi, i, tN, wN);
    for (int i = threadIdx.x; i < n_theta; i += blockDim.x) legendre_root(n_theta, i, tM, wM);
    __syncthreads();
    const int L = n_phi * n_theta;
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        const int n = l / n_theta, m = l % n_theta;
        const double phi = (1.0 + tN[n]) * kPi / 2.0;
        const double th = (1.0 + tM[m]) * kPi / 2.0;
        double sp, cp, st, ct;
        sincos(phi, &sp, &cp);
        sincos(th, &st, &ct);
        const dbl4 d = {sp * ct, sp * st, cp, (kPi / 16.0) * sp * wN[n] * wM[m]};
        f64[l] = d;
        f32[l] = make_float4((float)d.x, (float)d.y, (float)d.z, (float)d.w);
    }
}

__global__ void tet_rule_kernel(int order, double *bary, double *w)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (order == 1) {
        for (int i = 0; i < 4; ++i) bary[i] = 0.25;
        w[0] = 1.0;
        return;
    }
    if (order == 4) {
        const double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0, b = (5.0 - sqrt(5.0)) / 20.0;
        for (int q = 0; q < 4; ++q) {
            for (int i = 0; i < 4; ++i) bary[4 * q + i] = (i == q) ? a : b;
            w[q] = 0.25;
        }
        return;
    }
    const int k = order == 8 ? 2 : order == 27 ? 3 : 4;
    double x[3][4], wt[3][4];  // alpha = 2 (u), 1 (v), 0 (t)
    for (int d = 0; d < 3; ++d) {
        const double a = 2.0 - d;
        jacobi_roots(k, a, x[d]);
        for (int i = 0; i < k; ++i) {
            const double dp = jacobi_dp(k, a, x[d][i]);
            wt[d][i] = 1.0 / ((1.0 - x[d][i] * x[d][i]) * dp * dp);  // [0,1] weight for (1-u)^a
            x[d][i] = 0.5 * (x[d][i] + 1.0);
        }
    }
    int q = 0;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j)
            for (int l = 0; l < k; ++l) {
                const double u = x[0][i], v = x[1][j], t = x[2][l];
                const double x1 = u, x2 = (1.0 - u) * v, x3 = (1.0 - u) * (1.0 - v) * t;
                bary[4 * q + 0] = 1.0 - x1 - x2 - x3;
                bary[4 * q + 1] = x1;
                bary[4 * q + 2] = x2;
                bary[4 * q + 3] = x3;
                w[q] = 6.0 * wt[0][i] * wt[1][j] * wt[2][l];
                ++q;
            }
}

}  // namespace

cudaError_t build_lines(int n_phi, int n_theta, float4 *f32, dbl4 *f64, cudaStream_t st)
{
    lines_kernel<<<1, 512, 0, st>>>(n_phi, n_theta, f32, f64);
    return cudaGetLastError();
}

cudaError_t build_tet_rule(int order, double *bary, double *w, cudaStream_t st)
{
    tet_rule_kernel<<<1, 32, 0, st>>>(order, bary, w);
    return cudaGetLastError();
}

}  // namespace bs
