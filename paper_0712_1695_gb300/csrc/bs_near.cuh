// bs_near.cuh -- device helpers shared by the velocity kernels (bs_velocity.cu) and the
// all-ray kernel (bs_ray.cu): tolerances of the ray rule, mbarrier / bulk-copy wrappers,
// small vectors, and the float64 form of the ray rule for one (point, tet) pair.
#pragma once

#include <math.h>

#include "bs_internal.cuh"

namespace bs {
namespace {

constexpr float kBoundPadF = 1e-4f;  // relative safety on the bounding-sphere line test
constexpr double kBoundPadD = 1e-9;
constexpr double kTau = 1e-9;        // chord length threshold, in units of the longest edge
constexpr float kDegenA = 1e-5f;     // float32: |a_i| below this with x inside/on the tet -> float64 pair
// A line with |b_i| <= eps |g_i| (|s . n_i| <= eps) is parallel to face i: that face bounds nothing
// and the line is outside the tet when a_i < -eps (the oracle's Moller-Trumbore treats
// |det| <= 1e-12 |e1||e2| as parallel and accepts area coordinates down to -1e-12).
constexpr double kParD = 1e-12;
constexpr float kParF = 1e-6f;
constexpr float kVertexFallback = 1e-5f;
constexpr long long kWaitCap = 1LL << 26;  // default poll limit of a bulk-copy wait (about a second)

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy helpers (inline PTX, sm_90+ forms valid on sm_103a)
// ---------------------------------------------------------------------------
__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ inline void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ inline void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ inline void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Shared-memory load the compiler may not hoist or merge: the line loops read warp-uniform per-pair or
// per-tet values per line on purpose, so that they do not occupy registers across the loop.
__device__ __forceinline__ float4 lds4(const float4 *p)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(smem_u32(p)));
    return v;
}

// bounded wait: false when `cap` polls did not see the phase complete
__device__ inline bool mbar_wait(uint64_t *bar, uint32_t parity, long long cap)
{
    for (long long i = 0; i < cap; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// After a wait gave up: wait (bounded again) for the next completion of every stage, so that no bulk
// copy of this CTA can still be landing in its shared memory when the CTA exits.  A stage whose copy
// was never issued gives up after `cap` polls.
template <int S>
__device__ inline void mbar_drain(uint64_t *full, uint32_t phase, long long cap)
{
#pragma unroll 1
    for (int st = 0; st < S; ++st) mbar_wait(&full[st], (phase >> st) & 1u, cap);
}

// ---------------------------------------------------------------------------
// small vector helpers
// ---------------------------------------------------------------------------
template <typename T>
struct V3 {
    T x, y, z;
};
template <typename T>
__device__ inline V3<T> mk(T x, T y, T z) { return {x, y, z}; }
template <typename T>
__device__ inline T dot3(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

template <typename T>
__device__ inline T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The near/far decision of a (point, tet) pair (Section 1: the tet is far when the point lies beyond
// far_ratio circumradii of its centroid), with explicit round-to-nearest operations (no contraction), so
// that every kernel that takes it -- the far sweep, which leaves the near pairs out of its sums, and the
// near pass and the mesh walk, which evaluate them -- decides every pair the same way, bit for bit.  float32: the point
// x' and the centroid c' in the tile frame (x' = x_hi - o, as the far sweep forms it), c_rho2 = the far
// record's first float4 (c', rho^2); float64: global coordinates, c_rho2 = the record's first four.
__device__ __forceinline__ bool pair_is_near_f32(float xp, float yp, float zp, float4 c_rho2, float fr2)
{
    const float dx = __fsub_rn(xp, c_rho2.x), dy = __fsub_rn(yp, c_rho2.y), dz = __fsub_rn(zp, c_rho2.z);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    return !(d2 > __fmul_rn(fr2, c_rho2.w));
}
__device__ __forceinline__ bool pair_is_near_f64(double x, double y, double z, const double *c_rho2, double fr2)
{
    const double dx = __dsub_rn(x, c_rho2[0]), dy = __dsub_rn(y, c_rho2[1]), dz = __dsub_rn(z, c_rho2[2]);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return !(d2 > __dmul_rn(fr2, c_rho2[3]));
}
// Can a point of the ball (centre, radius) = sphere be near a tet of the tile (header: origin o and the
// radius rc of its centroids about o; rho_max its largest circumradius)?  No, when the ball is farther
// than far_ratio rho_max from every centroid, with a margin (0.1% and 1e-5 of the coordinates' scale)
// that covers the float32 rounding of this test and of the per-pair test: a culled tile holds no pair
// the per-pair test would call near.
__device__ __forceinline__ bool tile_culled(float4 sphere, float4 hdr, float rho_max, float far_ratio)
{
    const float dx = sphere.x - hdr.x, dy = sphere.y - hdr.y, dz = sphere.z - hdr.z;
    const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
    const float scale = fabsf(hdr.x) + fabsf(hdr.y) + fabsf(hdr.z) + dist;
    return dist - sphere.w - hdr.w > far_ratio * rho_max * 1.001f + 1e-5f * scale;
}

// Everything about a pair that does not depend on the line, in float64.
struct PairF64 {
    double a[4];           // lambda_i(x); exactly e_k when x is vertex k
    V3<double> g[4];       // face-plane gradients, g0 = -(g1 + g2 + g3)
    V3<double> w[4];       // nodal vorticity
    V3<double> Wa;         // omega interpolated (linearly extended) at x
    V3<double> rc;         // centroid - x
    double rc2, bound, tau_h, par2[4];
};

__device__ inline int vertex_index(V3<double> x, const double *__restrict__ r)
{
    int vk = -1;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (vk < 0 && r[nf64::V + 3 * i] == x.x && r[nf64::V + 3 * i + 1] == x.y && r[nf64::V + 3 * i + 2] == x.z)
            vk = i;
    return vk;
}

__device__ inline void pair_setup_f64(PairF64 &P, V3<double> x, const double *__restrict__ r, int vk)
{
    P.g[1] = mk(r[nf64::G + 0], r[nf64::G + 1], r[nf64::G + 2]);
    P.g[2] = mk(r[nf64::G + 3], r[nf64::G + 4], r[nf64::G + 5]);
    P.g[3] = mk(r[nf64::G + 6], r[nf64::G + 7], r[nf64::G + 8]);
    P.g[0] = mk(-(P.g[1].x + P.g[2].x + P.g[3].x), -(P.g[1].y + P.g[2].y + P.g[3].y),
                -(P.g[1].z + P.g[2].z + P.g[3].z));
#pragma unroll
    for (int i = 0; i < 4; ++i) P.w[i] = mk(r[nf64::W + 3 * i], r[nf64::W + 3 * i + 1], r[nf64::W + 3 * i + 2]);
    if (vk >= 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) P.a[i] = (i == vk) ? 1.0 : 0.0;
    } else {
        const V3<double> d0 = mk(x.x - r[nf64::V], x.y - r[nf64::V + 1], x.z - r[nf64::V + 2]);
        P.a[1] = dot3(P.g[1], d0);
        P.a[2] = dot3(P.g[2], d0);
        P.a[3] = dot3(P.g[3], d0);
        P.a[0] = 1.0 - P.a[1] - P.a[2] - P.a[3];
    }
    const double *a = P.a;
    P.Wa = mk(a[0] * P.w[0].x + a[1] * P.w[1].x + a[2] * P.w[2].x + a[3] * P.w[3].x,
              a[0] * P.w[0].y + a[1] * P.w[1].y + a[2] * P.w[2].y + a[3] * P.w[3].y,
              a[0] * P.w[0].z + a[1] * P.w[1].z + a[2] * P.w[2].z + a[3] * P.w[3].z);
    P.rc = mk(r[nf64::C] - x.x, r[nf64::C + 1] - x.y, r[nf64::C + 2] - x.z);
    P.rc2 = dot3(P.rc, P.rc);
    P.bound = r[nf64::RB2] * (1.0 + kBoundPadD);
    P.tau_h = kTau * r[nf64::H];
#pragma unroll
    for (int i = 0; i < 4; ++i) P.par2[i] = kParD * kParD * dot3(P.g[i], P.g[i]);
}

// One line in float64; adds k * s x J to acc and returns true on a hit.
__device__ inline bool line_f64(const PairF64 &P, const dbl4 ln, V3<double> &acc)
{
    const V3<double> s = mk(ln.x, ln.y, ln.z);
    const double rs = dot3(P.rc, s);
    if (P.rc2 - rs * rs > P.bound) return false;  // line farther than Rb from the centroid
    double b[4];
    b[1] = dot3(P.g[1], s);
    b[2] = dot3(P.g[2], s);
    b[3] = dot3(P.g[3], s);
    b[0] = -(b[1] + b[2] + b[3]);
    double lo = -INFINITY, hi = INFINITY;
    bool empty = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (b[i] * b[i] <= P.par2[i]) empty = empty || (P.a[i] < -kParD);
        else if (b[i] > 0.0) lo = fmax(lo, -P.a[i] / b[i]);
        else hi = fmin(hi, -P.a[i] / b[i]);
    }
    if (empty || !(hi - lo > P.tau_h)) return false;
    const V3<double> *w = P.w;
    const V3<double> Wb = mk(b[0] * w[0].x + b[1] * w[1].x + b[2] * w[2].x + b[3] * w[3].x,
                             b[0] * w[0].y + b[1] * w[1].y + b[2] * w[2].y + b[3] * w[3].y,
                             b[0] * w[0].z + b[1] * w[1].z + b[2] * w[2].z + b[3] * w[3].z);
    const double f1 = fabs(hi) - fabs(lo);
    const double f2 = 0.5 * (hi * fabs(hi) - lo * fabs(lo));
    const V3<double> J = mk(f1 * P.Wa.x + f2 * Wb.x, f1 * P.Wa.y + f2 * Wb.y, f1 * P.Wa.z + f2 * Wb.z);
    acc.x += ln.w * (s.y * J.z - s.z * J.y);
    acc.y += ln.w * (s.z * J.x - s.x * J.z);
    acc.z += ln.w * (s.x * J.y - s.y * J.x);
    return true;
}

// One line in float64 with the record read from memory as it is needed (a
// small register footprint: used for the rare float64 steps of the float32
// path).  vk = vertex index of x in the tet or -1.
__device__ __noinline__ bool line_f64_lean(V3<double> x, const double *__restrict__ r, int vk, const dbl4 ln,
                                           V3<double> &acc)
{
    const V3<double> s = mk(ln.x, ln.y, ln.z);
    {
        const V3<double> rc = mk(r[nf64::C] - x.x, r[nf64::C + 1] - x.y, r[nf64::C + 2] - x.z);
        const double rs = dot3(rc, s);
        if (dot3(rc, rc) - rs * rs > r[nf64::RB2] * (1.0 + kBoundPadD)) return false;
    }
    double a[4], b[4];
    {
        const V3<double> d0 = mk(x.x - r[nf64::V], x.y - r[nf64::V + 1], x.z - r[nf64::V + 2]);
        double sa = 0.0, sb = 0.0;
        for (int i = 1; i < 4; ++i) {
            const V3<double> g = mk(r[nf64::G + 3 * i - 3], r[nf64::G + 3 * i - 2], r[nf64::G + 3 * i - 1]);
            a[i] = dot3(g, d0);
            b[i] = dot3(g, s);
            sa += a[i];
            sb += b[i];
        }
        a[0] = 1.0 - sa;
        b[0] = -sb;
        if (vk >= 0)
            for (int i = 0; i < 4; ++i) a[i] = (i == vk) ? 1.0 : 0.0;
    }
    double lo = -INFINITY, hi = INFINITY;
    bool empty = false;
    for (int i = 0; i < 4; ++i) {
        V3<double> g;
        if (i == 0) {
            g = mk(0.0, 0.0, 0.0);
            for (int j = 1; j < 4; ++j) {
                g.x -= r[nf64::G + 3 * j - 3];
                g.y -= r[nf64::G + 3 * j - 2];
                g.z -= r[nf64::G + 3 * j - 1];
            }
        } else {
            g = mk(r[nf64::G + 3 * i - 3], r[nf64::G + 3 * i - 2], r[nf64::G + 3 * i - 1]);
        }
        if (b[i] * b[i] <= kParD * kParD * dot3(g, g)) empty = empty || (a[i] < -kParD);
        else if (b[i] > 0.0) lo = fmax(lo, -a[i] / b[i]);
        else hi = fmin(hi, -a[i] / b[i]);
    }
    if (empty || !(hi - lo > kTau * r[nf64::H])) return false;
    const double f1 = fabs(hi) - fabs(lo);
    const double f2 = 0.5 * (hi * fabs(hi) - lo * fabs(lo));
    V3<double> J = mk(0.0, 0.0, 0.0);
    for (int i = 0; i < 4; ++i) {
        const double c = f1 * a[i] + f2 * b[i];
        J.x += c * r[nf64::W + 3 * i];
        J.y += c * r[nf64::W + 3 * i + 1];
        J.z += c * r[nf64::W + 3 * i + 2];
    }
    acc.x += ln.w * (s.y * J.z - s.z * J.y);
    acc.y += ln.w * (s.z * J.x - s.x * J.z);
    acc.z += ln.w * (s.x * J.y - s.y * J.x);
    return true;
}

// The same, inlined (the lean drain of the velocity kernel runs it where little else is live).
__device__ __forceinline__ bool line_f64_lean_inl(V3<double> x, const double *__restrict__ r, int vk, const dbl4 ln,
                                           V3<double> &acc)
{
    const V3<double> s = mk(ln.x, ln.y, ln.z);
    {
        const V3<double> rc = mk(r[nf64::C] - x.x, r[nf64::C + 1] - x.y, r[nf64::C + 2] - x.z);
        const double rs = dot3(rc, s);
        if (dot3(rc, rc) - rs * rs > r[nf64::RB2] * (1.0 + kBoundPadD)) return false;
    }
    double a[4], b[4];
    {
        const V3<double> d0 = mk(x.x - r[nf64::V], x.y - r[nf64::V + 1], x.z - r[nf64::V + 2]);
        double sa = 0.0, sb = 0.0;
        for (int i = 1; i < 4; ++i) {
            const V3<double> g = mk(r[nf64::G + 3 * i - 3], r[nf64::G + 3 * i - 2], r[nf64::G + 3 * i - 1]);
            a[i] = dot3(g, d0);
            b[i] = dot3(g, s);
            sa += a[i];
            sb += b[i];
        }
        a[0] = 1.0 - sa;
        b[0] = -sb;
        if (vk >= 0)
            for (int i = 0; i < 4; ++i) a[i] = (i == vk) ? 1.0 : 0.0;
    }
    double lo = -INFINITY, hi = INFINITY;
    bool empty = false;
    for (int i = 0; i < 4; ++i) {
        V3<double> g;
        if (i == 0) {
            g = mk(0.0, 0.0, 0.0);
            for (int j = 1; j < 4; ++j) {
                g.x -= r[nf64::G + 3 * j - 3];
                g.y -= r[nf64::G + 3 * j - 2];
                g.z -= r[nf64::G + 3 * j - 1];
            }
        } else {
            g = mk(r[nf64::G + 3 * i - 3], r[nf64::G + 3 * i - 2], r[nf64::G + 3 * i - 1]);
        }
        if (b[i] * b[i] <= kParD * kParD * dot3(g, g)) empty = empty || (a[i] < -kParD);
        else if (b[i] > 0.0) lo = fmax(lo, -a[i] / b[i]);
        else hi = fmin(hi, -a[i] / b[i]);
    }
    if (empty || !(hi - lo > kTau * r[nf64::H])) return false;
    const double f1 = fabs(hi) - fabs(lo);
    const double f2 = 0.5 * (hi * fabs(hi) - lo * fabs(lo));
    V3<double> J = mk(0.0, 0.0, 0.0);
    for (int i = 0; i < 4; ++i) {
        const double c = f1 * a[i] + f2 * b[i];
        J.x += c * r[nf64::W + 3 * i];
        J.y += c * r[nf64::W + 3 * i + 1];
        J.z += c * r[nf64::W + 3 * i + 2];
    }
    acc.x += ln.w * (s.y * J.z - s.z * J.y);
    acc.y += ln.w * (s.z * J.x - s.x * J.z);
    acc.z += ln.w * (s.x * J.y - s.y * J.x);
    return true;
}

}  // namespace
}  // namespace bs
