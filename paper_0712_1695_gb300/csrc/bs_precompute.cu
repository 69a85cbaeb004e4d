// bs_precompute.cu -- per-tet tables, one thread per tet, float64 arithmetic.
//
// Near record (parameter independent, Section 2.1): the face planes of the
// tet as barycentric gradients g_i, so that along the line x + t s
//   lambda_i(t) = a_i + b_i t,  a_i = lambda_i(x),  b_i = g_i . s,
// plus the nodal vorticity (linear over the tet, Section 2), the longest edge
// h (chord threshold and the paper's pre-check scale), the centroid c and the
// bounding radius Rb about it (a line farther than Rb from c misses the tet).
//
// Far record (per tet rule and tile size): centroid, circumradius^2 (near/far
// test) and, per quadrature point, x_q and w'_q = -(w_q |V| / 4pi) omega(x_q),
// so that the far rule of Eq. 1 is v += sum_q (x - x_q) x w'_q / |x - x_q|^3.
#include <math.h>

#include "bs_internal.cuh"

namespace bs {
namespace {

struct D3 {
    double x, y, z;
};
__device__ inline D3 sub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ inline double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline D3 cross(D3 a, D3 b)
{
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ inline D3 scale(D3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ inline D3 load3(const double *p) { return {p[0], p[1], p[2]}; }

__global__ void near_records_kernel(const double *__restrict__ nodes, int64_t n_nodes,
                                    const int32_t *__restrict__ tets, int64_t n_tets,
                                    const double *__restrict__ omega, float4 *__restrict__ near32,
                                    double *__restrict__ near64, double *__restrict__ rho2, int *flag,
                                    unsigned long long *first_bad)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_tets) return;
    int32_t id[4];
    bool ok = true;
    for (int i = 0; i < 4; ++i) {
        id[i] = tets[4 * e + i];
        ok = ok && id[i] >= 0 && id[i] < n_nodes;
    }
    double *r = near64 + e * kNearF64;
    if (!ok) {
        atomicOr(flag, kFlagMeshIndex);
        atomicMin(first_bad, (unsigned long long)e);
        for (int i = 0; i < kNearF64; ++i) r[i] = 0.0;
        for (int i = 0; i < kNearF32Vec4; ++i) near32[e * kNearF32Vec4 + i] = make_float4(0.f, 0.f, 0.f, 0.f);
        rho2[e] = 0.0;
        return;
    }
    D3 v[4], w[4];
    for (int i = 0; i < 4; ++i) {
        v[i] = load3(nodes + 3 * (int64_t)id[i]);
        w[i] = load3(omega + 3 * (int64_t)id[i]);
    }
    const D3 e1 = sub(v[1], v[0]), e2 = sub(v[2], v[0]), e3 = sub(v[3], v[0]);
    const D3 n1 = cross(e2, e3), n2 = cross(e3, e1), n3 = cross(e1, e2);
    const double V6 = dot(e1, n1);
    double h2 = 0.0;
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b) {
            const D3 d = sub(v[b], v[a]);
            h2 = fmax(h2, dot(d, d));
        }
    const double h = sqrt(h2);
    if (!(fabs(V6) / 6.0 > 1e-14 * h2 * h)) {
        atomicOr(flag, kFlagMeshVolume);
        atomicMin(first_bad, (unsigned long long)e);
    }
    const double inv = 1.0 / V6;
    const D3 g1 = scale(n1, inv), g2 = scale(n2, inv), g3 = scale(n3, inv);
    const D3 c = scale({v[0].x + v[1].x + v[2].x + v[3].x, v[0].y + v[1].y + v[2].y + v[3].y,
                        v[0].z + v[1].z + v[2].z + v[3].z}, 0.25);
    // circumcentre relative to v0: p' = (|e1|^2 n1 + |e2|^2 n2 + |e3|^2 n3) / (2 V6)
    const double l1 = dot(e1, e1), l2 = dot(e2, e2), l3 = dot(e3, e3);
    const D3 pc = scale({l1 * n1.x + l2 * n2.x + l3 * n3.x, l1 * n1.y + l2 * n2.y + l3 * n3.y,
                         l1 * n1.z + l2 * n2.z + l3 * n3.z}, 0.5 * inv);
    rho2[e] = dot(pc, pc);
    double rb2 = 0.0;
    for (int i = 0; i < 4; ++i) {
        const D3 d = sub(v[i], c);
        rb2 = fmax(rb2, dot(d, d));
    }
    // float64 record
    for (int i = 0; i < 4; ++i) {
        r[nf64::V + 3 * i + 0] = v[i].x;
        r[nf64::V + 3 * i + 1] = v[i].y;
        r[nf64::V + 3 * i + 2] = v[i].z;
        r[nf64::W + 3 * i + 0] = w[i].x;
        r[nf64::W + 3 * i + 1] = w[i].y;
        r[nf64::W + 3 * i + 2] = w[i].z;
    }
    const D3 g[3] = {g1, g2, g3};
    for (int i = 0; i < 3; ++i) {
        r[nf64::G + 3 * i + 0] = g[i].x;
        r[nf64::G + 3 * i + 1] = g[i].y;
        r[nf64::G + 3 * i + 2] = g[i].z;
    }
    r[nf64::C + 0] = c.x;
    r[nf64::C + 1] = c.y;
    r[nf64::C + 2] = c.z;
    r[nf64::H] = h;
    r[nf64::RB2] = rb2;
    r[38] = 0.0;
    r[39] = 0.0;
    // float32 record (layout in bs_internal.cuh)
    float4 *f = near32 + e * kNearF32Vec4;
    f[nf32::G1] = make_float4((float)g1.x, (float)g1.y, (float)g1.z, (float)h);
    f[nf32::G2] = make_float4((float)g2.x, (float)g2.y, (float)g2.z, (float)rb2);
    f[nf32::G3] = make_float4((float)g3.x, (float)g3.y, (float)g3.z, 0.f);
    for (int i = 0; i < 4; ++i) f[nf32::W + i] = make_float4((float)w[i].x, (float)w[i].y, (float)w[i].z, 0.f);
    float hi[3], mid[3], lo;
    const double cc[3] = {c.x, c.y, c.z};
    for (int j = 0; j < 3; ++j) split3(cc[j], hi[j], mid[j], lo);
    f[nf32::CH] = make_float4(hi[0], hi[1], hi[2], 0.f);
    f[nf32::CM] = make_float4(mid[0], mid[1], mid[2], 0.f);
    float *vh = reinterpret_cast<float *>(f + nf32::VH), *vm = reinterpret_cast<float *>(f + nf32::VM);
    for (int i = 0; i < 4; ++i) {
        const double vv[3] = {v[i].x, v[i].y, v[i].z};
        for (int j = 0; j < 3; ++j) split3(vv[j], vh[3 * i + j], vm[3 * i + j], lo);
    }
}

// Tile headers, one thread per tile of `tile` consecutive tets, two float4:
// [origin o (mean of the centroids, rounded to float), radius rc of the
// centroids about o (rounded up)] [largest circumradius, 0, 0, 0].  A point x is far from every
// tet of the tile when |x - o| - rc > far_ratio * rho_max.
__global__ void tile_headers_kernel(const double *__restrict__ near64, const double *__restrict__ rho2,
                                    int64_t n_tets, int tile, float4 *__restrict__ hdr)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t first = t * tile;
    if (first >= n_tets) return;
    const int cnt = (int)min((int64_t)tile, n_tets - first);
    D3 o = {0, 0, 0};
    double rmax = 0.0;
    for (int j = 0; j < cnt; ++j) {
        const D3 c = load3(near64 + (first + j) * kNearF64 + nf64::C);
        o = {o.x + c.x, o.y + c.y, o.z + c.z};
        rmax = fmax(rmax, rho2[first + j]);
    }
    o = scale(o, 1.0 / cnt);
    const float ox = (float)o.x, oy = (float)o.y, oz = (float)o.z;
    const D3 of = {(double)ox, (double)oy, (double)oz};
    double rc = 0.0;
    for (int j = 0; j < cnt; ++j) {
        const D3 d = sub(load3(near64 + (first + j) * kNearF64 + nf64::C), of);
        rc = fmax(rc, sqrt(dot(d, d)));
    }
    hdr[2 * t] = make_float4(ox, oy, oz, (float)(rc * (1.0 + 1e-6) + 1e-30));
    hdr[2 * t + 1] = make_float4((float)(sqrt(rmax) * (1.0 + 1e-6)), 0.f, 0.f, 0.f);
}

// float32 far record (tile frame, x' = x - o of the tet's tile): [c' (3), rho^2] then per
// quadrature point the ten values [-2 x_q' (3), |x_q'|^2, w'_q (3), B_q (3)], with B_q = x_q' x w'_q,
// so that sum_q (x' - x_q') x w'_q / |x' - x_q'|^3 = x' x A - B with A = sum_q w'_q / r_q^3,
// B = sum_q B_q / r_q^3 and r_q^2 = |x'|^2 - 2 x'.x_q' + |x_q'|^2 (small terms in the tile frame).
// Quadrature-pair layout: value k of point q at float 4 + 20 (q / 2) + 2k + (q % 2); point-pair layout:
// at floats 4 + 20 q + 2k and 4 + 20 q + 2k + 1 (twice).
// float64 far record: [c (3), rho^2] then per q the same ten values.
__global__ void far_records_kernel(const double *__restrict__ near64, const double *__restrict__ rho2,
                                   int64_t n_tets, int Q, int tile, int layout, const double *__restrict__ bary,
                                   const double *__restrict__ wq, const float4 *__restrict__ hdr,
                                   float *__restrict__ far32, double *__restrict__ far64)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_tets) return;
    const double *r = near64 + e * kNearF64;
    D3 v[4], w[4];
    for (int i = 0; i < 4; ++i) {
        v[i] = load3(r + nf64::V + 3 * i);
        w[i] = load3(r + nf64::W + 3 * i);
    }
    const double vol = fabs(dot(sub(v[1], v[0]), cross(sub(v[2], v[0]), sub(v[3], v[0])))) / 6.0;
    const int s32 = far_stride<float>(Q, layout), s64 = far_stride<double>(Q);
    float *f = far32 + e * s32;
    double *d = far64 + e * s64;
    const float4 h = hdr[2 * (e / tile)];
    const D3 o = {(double)h.x, (double)h.y, (double)h.z};
    const D3 c = load3(r + nf64::C);
    d[0] = c.x;
    d[1] = c.y;
    d[2] = c.z;
    d[3] = rho2[e];
    const D3 cl = sub(c, o);
    f[0] = (float)cl.x;
    f[1] = (float)cl.y;
    f[2] = (float)cl.z;
    f[3] = (float)rho2[e];
    const double s = -vol / (4.0 * kPi);
    for (int q = 0; q < Q; ++q) {
        D3 xq = {0, 0, 0}, wv = {0, 0, 0};
        for (int i = 0; i < 4; ++i) {
            const double b = bary[4 * q + i];
            xq = {xq.x + b * v[i].x, xq.y + b * v[i].y, xq.z + b * v[i].z};
            wv = {wv.x + b * w[i].x, wv.y + b * w[i].y, wv.z + b * w[i].z};
        }
        wv = scale(wv, s * wq[q]);
        const D3 xl = sub(xq, o);
        const D3 B = cross(xl, wv);
        // float64: the same tile-frame values, one point after the other
        const double vals[10] = {-2.0 * xl.x, -2.0 * xl.y, -2.0 * xl.z, dot(xl, xl), wv.x, wv.y, wv.z, B.x, B.y, B.z};
        for (int j = 0; j < 10; ++j) d[4 + 10 * q + j] = vals[j];
        if (layout == kFarPointPairs) {
            float *g = f + 4 + 20 * q;
            for (int k = 0; k < 10; ++k) g[2 * k] = g[2 * k + 1] = (float)vals[k];
        } else {
            // pair q/2, slot q%2: value k of the point goes to float 2k + slot of the pair's 20
            float *g = f + 4 + 20 * (q / 2) + (q % 2);
            for (int k = 0; k < 10; ++k) g[2 * k] = (float)vals[k];
        }
    }
    if (layout == kFarQuadPairs && Q % 2) {
        // pad the last pair with a point of zero weight (|x - x_q| = sqrt(|x'|^2 + 1) > 0)
        float *g = f + 4 + 20 * (Q / 2) + 1;
        for (int k = 0; k < 10; ++k) g[2 * k] = (k == 3) ? 1.0f : 0.0f;
    }
}

}  // namespace

cudaError_t build_near_records(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                               const double *omega, float4 *near32, double *near64, double *rho2, int *flag,
                               unsigned long long *first_bad, cudaStream_t st)
{
    if (n_tets == 0) return cudaSuccess;
    const int tb = 128;
    near_records_kernel<<<(unsigned)((n_tets + tb - 1) / tb), tb, 0, st>>>(nodes, n_nodes, tets, n_tets, omega,
                                                                          near32, near64, rho2, flag, first_bad);
    return cudaGetLastError();
}

cudaError_t build_far_records(const double *near64, const double *rho2, int64_t n_tets, const TetRule &rule,
                              int tile, int layout32, float4 *hdr, float *far32, double *far64, cudaStream_t st)
{
    if (n_tets == 0) return cudaSuccess;
    const int tb = 128;
    const int64_t n_tiles = (n_tets + tile - 1) / tile;
    tile_headers_kernel<<<(unsigned)((n_tiles + tb - 1) / tb), tb, 0, st>>>(near64, rho2, n_tets, tile, hdr);
    far_records_kernel<<<(unsigned)((n_tets + tb - 1) / tb), tb, 0, st>>>(near64, rho2, n_tets, rule.order, tile,
                                                                         layout32, rule.bary, rule.w, hdr, far32,
                                                                         far64);
    return cudaGetLastError();
}

}  // namespace bs
