// Exact integral of Eq. 1 over one tetrahedron with linear vorticity (float64 geometry): the analytic near-field
// evaluation that Section 1 sets the ray rule against (the reduction of the volume integral to face
// integrals and then to closed-form edge integrals).
//
// With R = x - y, rho = |R|, the integrand is R x omega / rho^3 = grad_y(1/rho) x omega
// = curl_y(omega/rho) - (curl omega)/rho, and curl omega is constant on a tet with linear omega.  The
// divergence theorem (n_f the outward unit normal of face f) gives
//   v(x) = -(1/4pi) [ sum_f n_f x int_f omega/rho dS - (curl omega) int_T 1/rho dV ],
//   int_T 1/rho dV = 1/2 sum_f h_f int_f 1/rho dS,   h_f = n_f . (y - x) on face f.
// Writing omega(y) = omega(x) + G (y - x) (G = grad omega) and p_f = x + h_f n_f,
//   int_f omega/rho dS = omega(x) I0_f + G (Ip_f + h_f n_f I0_f),
//   I0_f = int_f 1/rho dS,   Ip_f = int_f (y - p_f)/rho dS,
// and the in-plane divergence theorem turns both into sums over the face's edges.  Per edge (unit
// tangent t from vertex a to vertex b, l = (y - x) . t along it, R0 = distance from x to the edge's line,
// R_a, R_b the distances to its ends, f = int dl / rho):
//   Ip_f += m E / 2,             E = R0^2 f + l_b R_b - l_a R_a,
//   I0_f += P0 f - |h_f| beta,   beta = atan(P0 l_b / (R0^2 + |h_f| R_b)) - atan(P0 l_a / (R0^2 + |h_f| R_a)),
// with m the edge's in-plane normal pointing out of the face and P0 = (a - x) . m.  f and E depend on the
// edge alone, so the 6 logarithms are shared by the two faces of each edge, and each difference of arc
// tangents is one atan2: atan(u) - atan(w) = arg((1 + iu)(1 - iw)) = atan2(u - w, 1 + uw), exact because
// both angles lie in (-pi/2, pi/2).  f takes the form free of cancellation for the signs of l_a, l_b; an
// edge whose line passes through x (R0 = 0) contributes nothing (P0 f and R0^2 f vanish there), and
// beta is dropped when P0 = 0.  With D = R0^2 + |h_f| R > 0 at both ends, the two arguments of atan2 are
// multiplied by D_a D_b, which removes every division from beta.
#pragma once

#include "bs_internal.cuh"
#include "bs_near.cuh"

namespace bs {

struct Vel64 {
    double x, y, z;
};

// v: contribution of the tet of near record r to the velocity at x.  LOWT: the logarithms and arc tangents
// in float32 (the geometry stays float64; about 1e-7 relative error per pair, for the float32 path); else
// every step in float64.
template <bool LOWT>
__device__ __noinline__ Vel64 tet_exact(const V3<double> x, const double *__restrict__ r)
{
    // vertices relative to x and their distances
    double dx[4], dy[4], dz[4], R[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        dx[i] = r[nf64::V + 3 * i] - x.x;
        dy[i] = r[nf64::V + 3 * i + 1] - x.y;
        dz[i] = r[nf64::V + 3 * i + 2] - x.z;
        R[i] = sqrt(dx[i] * dx[i] + dy[i] * dy[i] + dz[i] * dz[i]);
    }
    // barycentric gradients g_1..g_3 from the record, g_0 = -(g_1 + g_2 + g_3)
    double gx[4], gy[4], gz[4];
#pragma unroll
    for (int i = 1; i < 4; ++i) {
        gx[i] = r[nf64::G + 3 * (i - 1)];
        gy[i] = r[nf64::G + 3 * (i - 1) + 1];
        gz[i] = r[nf64::G + 3 * (i - 1) + 2];
    }
    gx[0] = -(gx[1] + gx[2] + gx[3]);
    gy[0] = -(gy[1] + gy[2] + gy[3]);
    gz[0] = -(gz[1] + gz[2] + gz[3]);
    // G[a][b] = d omega_a / d y_b = sum_i (omega_i - omega_0)_a g_i,b
    double G[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double w0 = r[nf64::W + a];
        const double w1 = r[nf64::W + 3 + a] - w0, w2 = r[nf64::W + 6 + a] - w0, w3 = r[nf64::W + 9 + a] - w0;
        G[a][0] = w1 * gx[1] + w2 * gx[2] + w3 * gx[3];
        G[a][1] = w1 * gy[1] + w2 * gy[2] + w3 * gy[3];
        G[a][2] = w1 * gz[1] + w2 * gz[2] + w3 * gz[3];
    }
    // omega(x) = omega_0 + G (x - v_0) = omega_0 - G d_0
    double wx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        wx[a] = r[nf64::W + a] - (G[a][0] * dx[0] + G[a][1] * dy[0] + G[a][2] * dz[0]);

    // edge terms: f = int dl / rho and E = R0^2 f + l_b R_b - l_a R_a
    constexpr int EA[6] = {0, 0, 0, 1, 1, 2}, EB[6] = {1, 2, 3, 2, 3, 3};
    double f[6], E[6], R02[6], IL[6];
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const int a = EA[e], b = EB[e];
        const double ex = dx[b] - dx[a], ey = dy[b] - dy[a], ez = dz[b] - dz[a];
        const double L2 = ex * ex + ey * ey + ez * ez, iL = rsqrt(L2);
        IL[e] = iL;
        const double tx = ex * iL, ty = ey * iL, tz = ez * iL;
        const double la = dx[a] * tx + dy[a] * ty + dz[a] * tz, lb = dx[b] * tx + dy[b] * ty + dz[b] * tz;
        const double cx = dy[a] * tz - dz[a] * ty, cy = dz[a] * tx - dx[a] * tz, cz = dx[a] * ty - dy[a] * tx;
        const double r02 = cx * cx + cy * cy + cz * cz;  // squared distance from x to the edge's line
        double fe = 0.0;
        if (r02 > 1e-26 * L2) {
            // the ratio is at most about 1e26 (r02 > 1e-26 L^2): within float range
            const double q = la >= 0.0 ? (R[b] + lb) / (R[a] + la)
                                       : (lb <= 0.0 ? (R[a] - la) / (R[b] - lb) : (R[b] + lb) * (R[a] - la) / r02);
            if constexpr (LOWT)
                fe = (double)logf((float)q);
            else
                fe = log(q);
        }
        f[e] = fe;
        R02[e] = r02;
        E[e] = r02 * fe + lb * R[b] - la * R[a];
    }

    // faces: face k is opposite vertex k; its edges and, for each, the face's third vertex
    constexpr int FE[4][3] = {{3, 4, 5}, {1, 2, 5}, {0, 2, 4}, {0, 1, 3}};
    constexpr int FO[4][3] = {{3, 2, 1}, {3, 2, 0}, {3, 1, 0}, {2, 1, 0}};
    double Sx = 0.0, Sy = 0.0, Sz = 0.0, vol = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double gn = rsqrt(gx[k] * gx[k] + gy[k] * gy[k] + gz[k] * gz[k]);
        const double nx = -gx[k] * gn, ny = -gy[k] * gn, nz = -gz[k] * gn;  // outward: lambda_k grows inwards
        const int v0 = EA[FE[k][0]];  // a vertex of face k
        const double h = nx * dx[v0] + ny * dy[v0] + nz * dz[v0];
        const double ah = fabs(h);
        double I0 = 0.0, Ipx = 0.0, Ipy = 0.0, Ipz = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int e = FE[k][j], a = EA[e], b = EB[e], o = FO[k][j];
            const double iL = IL[e];
            const double tx = (dx[b] - dx[a]) * iL, ty = (dy[b] - dy[a]) * iL, tz = (dz[b] - dz[a]) * iL;
            // in-plane normal of the edge, pointing away from the face's third vertex
            double mx = ty * nz - tz * ny, my = tz * nx - tx * nz, mz = tx * ny - ty * nx;
            if (mx * (dx[o] - dx[a]) + my * (dy[o] - dy[a]) + mz * (dz[o] - dz[a]) > 0.0) {
                mx = -mx;
                my = -my;
                mz = -mz;
            }
            const double P0 = dx[a] * mx + dy[a] * my + dz[a] * mz;
            double beta = 0.0;
            if (fabs(P0) * iL > 1e-13) {
                // u - w and 1 + u w over the common positive factor Da Db (atan2 ignores it): no division
                const double la = dx[a] * tx + dy[a] * ty + dz[a] * tz, lb = dx[b] * tx + dy[b] * ty + dz[b] * tz;
                const double Da = R02[e] + ah * R[a], Db = R02[e] + ah * R[b];
                const double yy = P0 * (lb * Da - la * Db), xx = Da * Db + P0 * P0 * la * lb;
                if constexpr (LOWT) {
                    // atan2 ignores a common positive scale: bring both into float range first
                    const double m = fmax(fabs(yy), fabs(xx));
                    beta = m > 0.0 ? (double)atan2f((float)(yy / m), (float)(xx / m)) : 0.0;
                } else {
                    beta = atan2(yy, xx);
                }
            }
            I0 += P0 * f[e] - ah * beta;
            const double c = 0.5 * E[e];
            Ipx += c * mx;
            Ipy += c * my;
            Ipz += c * mz;
        }
        const double qx = Ipx + h * nx * I0, qy = Ipy + h * ny * I0, qz = Ipz + h * nz * I0;
        const double Iwx = wx[0] * I0 + G[0][0] * qx + G[0][1] * qy + G[0][2] * qz;
        const double Iwy = wx[1] * I0 + G[1][0] * qx + G[1][1] * qy + G[1][2] * qz;
        const double Iwz = wx[2] * I0 + G[2][0] * qx + G[2][1] * qy + G[2][2] * qz;
        Sx += ny * Iwz - nz * Iwy;
        Sy += nz * Iwx - nx * Iwz;
        Sz += nx * Iwy - ny * Iwx;
        vol += 0.5 * h * I0;
    }
    const double cx = G[2][1] - G[1][2], cy = G[0][2] - G[2][0], cz = G[1][0] - G[0][1];
    const double s = -0.25 / 3.14159265358979323846;
    return {s * (Sx - cx * vol), s * (Sy - cy * vol), s * (Sz - cz * vol)};
}

}  // namespace bs
