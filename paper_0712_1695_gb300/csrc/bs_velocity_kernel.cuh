// bs_velocity_kernel.cuh -- the velocity kernel (Eq. 1 by the far tet rule
// and the ray rule of Section 2), float32 and float64, as a template over its
// launch shape.  The bs_vel_*.cu files instantiate the variants (one file per
// precision / rule family, compiled in parallel); bs_velocity.cu selects and
// launches them.
//
// Work decomposition (N-body style, one GPU):
//   item = (block of P*NT evaluation points, chunk of consecutive tet tiles).
//   A persistent grid pulls items from a device counter.  Each CTA keeps its
//   points in registers (P per thread) and in shared memory, and streams the
//   chunk's far records tile by tile into a double-buffered shared-memory
//   ring with one bulk asynchronous copy (cp.async.bulk + mbarrier) per tile.
//   Every thread classifies its points against each tet of the tile (one
//   warp-uniform broadcast read of the record per tet); far pairs go through
//   the tet Gauss rule, near pairs are recorded in a per-warp queue as warp
//   ballot masks.  The queue is drained by the whole warp: the 32 lanes split
//   the n_theta*n_phi lines of one pair, and the three velocity components
//   are reduced with shuffles and handed to the lane that owns the point.
//   float32: per-tile partial sums in float32, Kahan-compensated across
//   tiles; each item writes its float64 partial to scratch[chunk][point]; a
//   second kernel adds the chunks in a fixed order (deterministic).
//
// Ray rule per line (Section 2.1, Eq. 5 with sign(R)): along x + t s the
// barycentric coordinates are lambda_i = a_i + b_i t; the chord is
// [lo, hi] = intersection of {a_i + b_i t >= 0}, and with omega = Wa + t Wb
// (Wa = sum a_i w_i, Wb = sum b_i w_i)
//   int_lo^hi sign(t) omega dt = (|hi| - |lo|) Wa + (hi|hi| - lo|lo|) Wb / 2,
// which equals Eq. 5's trapezoid (R1 - R0)(w0 + w1)/2 on each side of t = 0.
// This plane clipping gives the same chord as the paper's four
// Moller-Trumbore face tests with fewer operations (no edge vectors, no
// cross products per line).
#pragma once

#include <math.h>

#include <algorithm>
#include <type_traits>

#include "bs_internal.cuh"
#include "bs_exact.cuh"
#include "bs_near.cuh"

namespace bs {
namespace {

// packed float pairs (lo = first value, hi = second) and the f32x2 arithmetic of sm_100+
__device__ __forceinline__ unsigned long long pack2(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
// 1/sqrt(x) with subnormal inputs flushed: the far sweep's r^2 is never subnormal (a far pair
// is at least the far ratio times the tet radius apart) and a masked near pair may give inf,
// which the mask discards; the flush drops the subnormal rescaling around every evaluation.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float sum2(unsigned long long v)
{
    float a, b;
    unpack2(v, a, b);
    return a + b;
}

// ---------------------------------------------------------------------------
// Ray rule for one (point, tet) pair, lines split across the 32 lanes.
// Returns the warp-reduced contribution (all lanes) and the hit count.
// ---------------------------------------------------------------------------
struct NearOut {
    double vx, vy, vz;
    int hits;
};
struct NearOut32 {
    float vx, vy, vz;
    int hits;
};

// float64 version: every step in double.  Used by the float64 path and by
// pairs of the float32 path whose point lies on an edge or face of the tet.
__device__ __noinline__ NearOut near_pair_f64(V3<double> x, const double *__restrict__ r,
                                              const dbl4 *__restrict__ lines, int L, int lane)
{
    PairF64 P;
    pair_setup_f64(P, x, r, vertex_index(x, r));
    V3<double> acc = mk(0.0, 0.0, 0.0);
    int hits = 0;
    for (int l = lane; l < L; l += 32) hits += line_f64(P, lines[l], acc) ? 1 : 0;
    NearOut o;
    o.vx = warp_sum(acc.x);
    o.vy = warp_sum(acc.y);
    o.vz = warp_sum(acc.z);
    o.hits = warp_sum(hits);
    return o;
}

__device__ __noinline__ void line_fallback_f64(V3<double> x, const float *__restrict__ xs,
                                               const float4 *__restrict__ r32, const double *__restrict__ r64,
                                               const float4 *__restrict__ lines, const dbl4 *__restrict__ lines64,
                                               int L, int lane, int vk, bool whole_f64, V3<double> &acc, int &hits);

// float32 version.  The point, the centroid and the vertices are float
// splits (hi + mid + lo), so the differences x - v0 and c - x and the vertex
// test need no float64 arithmetic and a_i carries no error from the absolute
// coordinates.
// When x is vertex k of the tet, a = e_k exactly and the chord is decided by
// the signs of b_i on the three faces through x; a line with
// |b_i| <= 1e-5 |g_i| on one of them (nearly in that face plane, where the
// chord jumps with the sign) is recomputed in float64 in a second pass, after
// the float32 state is dead (keeps the register footprint of the pass
// small).  Pairs whose point is within 1e-5 (barycentric) of the tet's
// boundary without being a vertex run wholly in float64.
//
// U (the ray bundle): each lane takes U of its lines per iteration (lines l, l + 32, ..., l + 32 (U-1)),
// unrolled, so that their loads and clipping interleave.
//
// DEFER: the float64 steps are not taken here; *redo_out (warp-uniform) says the pair needs them, *vk_out and
// *whole_out how, and the caller runs line_fallback_f64_inl for it later (where few registers are live).
template <int U, bool DEFER = false>
__device__ __forceinline__ NearOut32 near_pair_f32_body(const float *__restrict__ xs, const float4 *__restrict__ r32,
                                                        const double *__restrict__ r64, const float4 *__restrict__ lines,
                                                        const dbl4 *__restrict__ lines64, int L, int lane,
                                                        bool *redo_out = nullptr, int *vk_out = nullptr,
                                                        bool *whole_out = nullptr)
{
    // xs: the point as float splits [component][hi, mid, lo]
    const float xh0 = xs[0], xm0 = xs[1], xh1 = xs[3], xm1 = xs[4], xh2 = xs[6], xm2 = xs[7];
    int vk = -1;
    {
        const float *vh = reinterpret_cast<const float *>(r32 + nf32::VH);
        const float *vm = reinterpret_cast<const float *>(r32 + nf32::VM);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (vk < 0 && vh[3 * i] == xh0 && vm[3 * i] == xm0 && vh[3 * i + 1] == xh1 && vm[3 * i + 1] == xm1 &&
                vh[3 * i + 2] == xh2 && vm[3 * i + 2] == xm2)
                vk = i;
    }
    float ax = 0.f, ay = 0.f, az = 0.f;
    int hits = 0;
    bool any_redo = false;
    bool whole_f64 = false;
    {
        const float4 q0 = r32[nf32::G1], q1 = r32[nf32::G2], q2 = r32[nf32::G3];
        V3<float> g[4];
        g[1] = mk(q0.x, q0.y, q0.z);
        g[2] = mk(q1.x, q1.y, q1.z);
        g[3] = mk(q2.x, q2.y, q2.z);
        g[0] = mk(-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z));
        const float h = q0.w, rb2 = q1.w;
        float a[4];
        if (vk >= 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = (i == vk) ? 1.0f : 0.0f;
        } else {
            // x - v0 from the splits: the hi parts are within a few tet sizes of each other
            const float *vh = reinterpret_cast<const float *>(r32 + nf32::VH);
            const float *vm = reinterpret_cast<const float *>(r32 + nf32::VM);
            const V3<float> d0 = mk((xh0 - vh[0]) + (xm0 - vm[0]), (xh1 - vh[1]) + (xm1 - vm[1]),
                                    (xh2 - vh[2]) + (xm2 - vm[2]));
            a[1] = dot3(g[1], d0);
            a[2] = dot3(g[2], d0);
            a[3] = dot3(g[3], d0);
            a[0] = 1.0f - a[1] - a[2] - a[3];
            const float amin = fminf(fminf(a[0], a[1]), fminf(a[2], a[3]));
            const float aabs = fminf(fminf(fabsf(a[0]), fabsf(a[1])), fminf(fabsf(a[2]), fabsf(a[3])));
            whole_f64 = amin > -kDegenA && aabs < kDegenA;
        }
        if (!whole_f64) {
            V3<float> w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 t = r32[nf32::W + i];
                w[i] = mk(t.x, t.y, t.z);
            }
            const V3<float> Wa = mk(a[0] * w[0].x + a[1] * w[1].x + a[2] * w[2].x + a[3] * w[3].x,
                                    a[0] * w[0].y + a[1] * w[1].y + a[2] * w[2].y + a[3] * w[3].y,
                                    a[0] * w[0].z + a[1] * w[1].z + a[2] * w[2].z + a[3] * w[3].z);
            const float4 ch = r32[nf32::CH], cm = r32[nf32::CM];
            const V3<float> rc = mk((ch.x - xh0) + (cm.x - xm0), (ch.y - xh1) + (cm.y - xm1), (ch.z - xh2) + (cm.z - xm2));
            const float rc2 = dot3(rc, rc);
            const float bound = rb2 * (1.0f + kBoundPadF);
            const float tau_h = (float)kTau * h;
            float par2[4], fb2[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float gg = dot3(g[i], g[i]);
                par2[i] = kParF * kParF * gg;
                // faces through vertex vk: below this |b_i| the sign is decided in float64
                fb2[i] = (vk >= 0 && i != vk) ? kVertexFallback * kVertexFallback * gg : -1.0f;
            }
            auto line = [&](const float4 ln) {
                const V3<float> s = mk(ln.x, ln.y, ln.z);
                const float rs = dot3(rc, s);
                if (rc2 - rs * rs > bound) return;
                float b[4];
                b[1] = dot3(g[1], s);
                b[2] = dot3(g[2], s);
                b[3] = dot3(g[3], s);
                b[0] = -(b[1] + b[2] + b[3]);
                bool redo = false;
#pragma unroll
                for (int i = 0; i < 4; ++i) redo = redo || (b[i] * b[i] <= fb2[i]);
                if (redo) {
                    any_redo = true;
                    return;
                }
                float lo = -INFINITY, hi = INFINITY;
                bool empty = false;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (b[i] * b[i] <= par2[i]) empty = empty || (a[i] < -kParF);
                    else if (b[i] > 0.f) lo = fmaxf(lo, -a[i] / b[i]);
                    else hi = fminf(hi, -a[i] / b[i]);
                }
                if (empty || !(hi - lo > tau_h)) return;
                const V3<float> Wb = mk(b[0] * w[0].x + b[1] * w[1].x + b[2] * w[2].x + b[3] * w[3].x,
                                        b[0] * w[0].y + b[1] * w[1].y + b[2] * w[2].y + b[3] * w[3].y,
                                        b[0] * w[0].z + b[1] * w[1].z + b[2] * w[2].z + b[3] * w[3].z);
                const float f1 = fabsf(hi) - fabsf(lo);
                const float f2 = 0.5f * (hi * fabsf(hi) - lo * fabsf(lo));
                const V3<float> J = mk(f1 * Wa.x + f2 * Wb.x, f1 * Wa.y + f2 * Wb.y, f1 * Wa.z + f2 * Wb.z);
                ax += ln.w * (s.y * J.z - s.z * J.y);
                ay += ln.w * (s.z * J.x - s.x * J.z);
                az += ln.w * (s.x * J.y - s.y * J.x);
                ++hits;
            };
#pragma unroll 1
            for (int l0 = lane; l0 < L; l0 += 32 * U) {
                float4 ln[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    ln[u] = (l0 + 32 * u < L) ? lines[l0 + 32 * u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (l0 + 32 * u < L) line(ln[u]);
            }
        }
    }
    if constexpr (DEFER) {
        *redo_out = whole_f64 || __any_sync(0xffffffffu, any_redo);
        *vk_out = vk;
        *whole_out = whole_f64;
    } else if (whole_f64 || any_redo) {
        // rare: lines (or whole pairs) that need float64; the point's exact coordinates from its splits
        V3<double> acc = mk(0.0, 0.0, 0.0);
        const V3<double> x = mk(join3(xs[0], xs[1], xs[2]), join3(xs[3], xs[4], xs[5]), join3(xs[6], xs[7], xs[8]));
        line_fallback_f64(x, xs, r32, r64, lines, lines64, L, lane, vk, whole_f64, acc, hits);
        ax += (float)acc.x;
        ay += (float)acc.y;
        az += (float)acc.z;
    }
    NearOut32 o;
    o.vx = warp_sum(ax);
    o.vy = warp_sum(ay);
    o.vz = warp_sum(az);
    o.hits = warp_sum(hits);
    return o;
}


// The lean form of near_pair_f32_body: the same ray rule, the same float64 fallbacks, but the
// pair's warp-uniform values (barycentric coordinates a_i of the point, the parallel and
// vertex-fallback thresholds, W_a, the centroid offset and the bounding test, g_0, the chord
// threshold) are written once to the warp's shared slot (kPairSlotVec4 float4) and read back per
// line, with the face gradients and nodal vorticity read from the staged near record.  The drain
// then holds only a line's temporaries in registers, so the kernel's far sweep keeps its registers.
constexpr int kPairSlotVec4 = 6;
// The pairs that need float64 steps (the point on an edge or face of the tet, or lines nearly in a face
// through the point's vertex) are not finished here: *redo is set (warp-uniform), *vk_out and *whole_out
// say how, and the caller runs line_fallback_f64_inl for the pair later.
template <int U>
__device__ __forceinline__ NearOut32 near_pair_f32_lean(const float *__restrict__ xs, const float4 *__restrict__ r32,
                                                        const float4 *__restrict__ lines, int L, int lane, float4 *slot,
                                                        bool *redo_out, int *vk_out, bool *whole_out)
{
    const float xh0 = xs[0], xm0 = xs[1], xh1 = xs[3], xm1 = xs[4], xh2 = xs[6], xm2 = xs[7];
    int vk = -1;
    {
        const float *vh = reinterpret_cast<const float *>(r32 + nf32::VH);
        const float *vm = reinterpret_cast<const float *>(r32 + nf32::VM);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (vk < 0 && vh[3 * i] == xh0 && vm[3 * i] == xm0 && vh[3 * i + 1] == xh1 && vm[3 * i + 1] == xm1 &&
                vh[3 * i + 2] == xh2 && vm[3 * i + 2] == xm2)
                vk = i;
    }
    float ax = 0.f, ay = 0.f, az = 0.f;
    int hits = 0;
    bool any_redo = false;
    bool whole_f64 = false;
    __syncwarp();  // every lane is done with the slot's previous pair
    {
        const float4 q0 = r32[nf32::G1], q1 = r32[nf32::G2], q2 = r32[nf32::G3];
        const V3<float> g1 = mk(q0.x, q0.y, q0.z), g2 = mk(q1.x, q1.y, q1.z), g3 = mk(q2.x, q2.y, q2.z);
        const V3<float> g0 = mk(-(g1.x + g2.x + g3.x), -(g1.y + g2.y + g3.y), -(g1.z + g2.z + g3.z));
        float a[4];
        if (vk >= 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = (i == vk) ? 1.0f : 0.0f;
        } else {
            const float *vh = reinterpret_cast<const float *>(r32 + nf32::VH);
            const float *vm = reinterpret_cast<const float *>(r32 + nf32::VM);
            const V3<float> d0 = mk((xh0 - vh[0]) + (xm0 - vm[0]), (xh1 - vh[1]) + (xm1 - vm[1]),
                                    (xh2 - vh[2]) + (xm2 - vm[2]));
            a[1] = dot3(g1, d0);
            a[2] = dot3(g2, d0);
            a[3] = dot3(g3, d0);
            a[0] = 1.0f - a[1] - a[2] - a[3];
            const float amin = fminf(fminf(a[0], a[1]), fminf(a[2], a[3]));
            const float aabs = fminf(fminf(fabsf(a[0]), fabsf(a[1])), fminf(fabsf(a[2]), fabsf(a[3])));
            whole_f64 = amin > -kDegenA && aabs < kDegenA;
        }
        if (!whole_f64 && lane == 0) {
            float wa[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 t = r32[nf32::W + i];
                wa[0] += a[i] * t.x;
                wa[1] += a[i] * t.y;
                wa[2] += a[i] * t.z;
            }
            const float4 ch = r32[nf32::CH], cm = r32[nf32::CM];
            const V3<float> rc = mk((ch.x - xh0) + (cm.x - xm0), (ch.y - xh1) + (cm.y - xm1), (ch.z - xh2) + (cm.z - xm2));
            const V3<float> gg[4] = {g0, g1, g2, g3};
            float par2[4], fb2[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float n2 = dot3(gg[i], gg[i]);
                par2[i] = kParF * kParF * n2;
                fb2[i] = (vk >= 0 && i != vk) ? kVertexFallback * kVertexFallback * n2 : -1.0f;
            }
            slot[0] = make_float4(a[0], a[1], a[2], a[3]);
            slot[1] = make_float4(par2[0], par2[1], par2[2], par2[3]);
            slot[2] = make_float4(fb2[0], fb2[1], fb2[2], fb2[3]);
            slot[3] = make_float4(wa[0], wa[1], wa[2], dot3(rc, rc));
            slot[4] = make_float4(rc.x, rc.y, rc.z, q1.w * (1.0f + kBoundPadF));
            slot[5] = make_float4(g0.x, g0.y, g0.z, (float)kTau * q0.w);
        }
    }
    __syncwarp();
    if (!whole_f64) {
        auto line = [&](const float4 ln) {
            const V3<float> s = mk(ln.x, ln.y, ln.z);
            const float4 rcb = lds4(slot + 4);
            const float rs = rcb.x * s.x + rcb.y * s.y + rcb.z * s.z;
            if (lds4(slot + 3).w - rs * rs > rcb.w) return;
            const float4 q0 = lds4(r32 + nf32::G1), q1 = lds4(r32 + nf32::G2), q2 = lds4(r32 + nf32::G3);
            const float4 gz = lds4(slot + 5);
            float b[4];
            b[1] = q0.x * s.x + q0.y * s.y + q0.z * s.z;
            b[2] = q1.x * s.x + q1.y * s.y + q1.z * s.z;
            b[3] = q2.x * s.x + q2.y * s.y + q2.z * s.z;
            b[0] = -(b[1] + b[2] + b[3]);
            const float4 f4 = lds4(slot + 2);
            const float fb2[4] = {f4.x, f4.y, f4.z, f4.w};
            bool redo = false;
#pragma unroll
            for (int i = 0; i < 4; ++i) redo = redo || (b[i] * b[i] <= fb2[i]);
            if (redo) {
                any_redo = true;
                return;
            }
            const float4 p4 = lds4(slot + 1), a4 = lds4(slot);
            const float par2[4] = {p4.x, p4.y, p4.z, p4.w}, a[4] = {a4.x, a4.y, a4.z, a4.w};
            float lo = -INFINITY, hi = INFINITY;
            bool empty = false;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (b[i] * b[i] <= par2[i]) empty = empty || (a[i] < -kParF);
                else if (b[i] > 0.f) lo = fmaxf(lo, -a[i] / b[i]);
                else hi = fminf(hi, -a[i] / b[i]);
            }
            if (empty || !(hi - lo > gz.w)) return;
            float Wb[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 t = lds4(r32 + nf32::W + i);
                Wb[0] += b[i] * t.x;
                Wb[1] += b[i] * t.y;
                Wb[2] += b[i] * t.z;
            }
            const float4 wa = lds4(slot + 3);
            const float f1 = fabsf(hi) - fabsf(lo);
            const float f2 = 0.5f * (hi * fabsf(hi) - lo * fabsf(lo));
            const V3<float> J = mk(f1 * wa.x + f2 * Wb[0], f1 * wa.y + f2 * Wb[1], f1 * wa.z + f2 * Wb[2]);
            ax += ln.w * (s.y * J.z - s.z * J.y);
            ay += ln.w * (s.z * J.x - s.x * J.z);
            az += ln.w * (s.x * J.y - s.y * J.x);
            ++hits;
        };
#pragma unroll 1
        for (int l0 = lane; l0 < L; l0 += 32 * U) {
            float4 ln[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                ln[u] = (l0 + 32 * u < L) ? lines[l0 + 32 * u] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (l0 + 32 * u < L) line(ln[u]);
        }
    }
    *redo_out = whole_f64 || __any_sync(0xffffffffu, any_redo);
    *vk_out = vk;
    *whole_out = whole_f64;
    NearOut32 o;
    o.vx = warp_sum(ax);
    o.vy = warp_sum(ay);
    o.vz = warp_sum(az);
    o.hits = warp_sum(hits);
    return o;
}

template <int U>
__device__ __noinline__ NearOut32 near_pair_f32(const float *__restrict__ xs, const float4 *__restrict__ r32,
                                                const double *__restrict__ r64, const float4 *__restrict__ lines,
                                                const dbl4 *__restrict__ lines64, int L, int lane)
{
    return near_pair_f32_body<U>(xs, r32, r64, lines, lines64, L, lane);
}

// The float64 steps of near_pair_f32 (kept out of line: they are rare, and their registers would
// otherwise count against the common path).
__device__ __noinline__ void line_fallback_f64(V3<double> x, const float *__restrict__ xs,
                                               const float4 *__restrict__ r32, const double *__restrict__ r64,
                                               const float4 *__restrict__ lines, const dbl4 *__restrict__ lines64,
                                               int L, int lane, int vk, bool whole_f64, V3<double> &acc, int &hits)
{
    const float xh0 = xs[0], xm0 = xs[1], xh1 = xs[3], xm1 = xs[4], xh2 = xs[6], xm2 = xs[7];
    if (whole_f64) {
#pragma unroll 1
        for (int l = lane; l < L; l += 32) hits += line_f64_lean(x, r64, -1, lines64[l], acc) ? 1 : 0;
    } else {
        // second pass: find this lane's flagged lines again (same float32 test) and redo them in float64
        const float4 q0 = r32[nf32::G1], q1 = r32[nf32::G2], q2 = r32[nf32::G3];
        const V3<float> g1 = mk(q0.x, q0.y, q0.z), g2 = mk(q1.x, q1.y, q1.z), g3 = mk(q2.x, q2.y, q2.z);
        const V3<float> g0 = mk(-(g1.x + g2.x + g3.x), -(g1.y + g2.y + g3.y), -(g1.z + g2.z + g3.z));
        const float4 ch = r32[nf32::CH], cm = r32[nf32::CM];
        const V3<float> rc = mk((ch.x - xh0) + (cm.x - xm0), (ch.y - xh1) + (cm.y - xm1), (ch.z - xh2) + (cm.z - xm2));
        const float rc2 = dot3(rc, rc), bound = q1.w * (1.0f + kBoundPadF);
        const float f = kVertexFallback * kVertexFallback;
#pragma unroll 1
        for (int l = lane; l < L; l += 32) {
            const float4 ln = lines[l];
            const V3<float> s = mk(ln.x, ln.y, ln.z);
            const float rs = dot3(rc, s);
            if (rc2 - rs * rs > bound) continue;
            const float b1 = dot3(g1, s), b2 = dot3(g2, s), b3 = dot3(g3, s), b0 = -(b1 + b2 + b3);
            const bool redo = (vk != 0 && b0 * b0 <= f * dot3(g0, g0)) || (vk != 1 && b1 * b1 <= f * dot3(g1, g1)) ||
                              (vk != 2 && b2 * b2 <= f * dot3(g2, g2)) || (vk != 3 && b3 * b3 <= f * dot3(g3, g3));
            if (redo && line_f64_lean(x, r64, vk, lines64[l], acc)) ++hits;
        }
    }
}

// The same float64 steps, inlined (with the float64 line routine inlined too): the lean drain runs them
// after a queue entry's pairs, where little else is live, instead of calling out from the pair routine.
__device__ __forceinline__ void line_fallback_f64_inl(V3<double> x, const float *__restrict__ xs,
                                               const float4 *__restrict__ r32, const double *__restrict__ r64,
                                               const float4 *__restrict__ lines, const dbl4 *__restrict__ lines64,
                                               int L, int lane, int vk, bool whole_f64, V3<double> &acc, int &hits)
{
    const float xh0 = xs[0], xm0 = xs[1], xh1 = xs[3], xm1 = xs[4], xh2 = xs[6], xm2 = xs[7];
    if (whole_f64) {
#pragma unroll 1
        for (int l = lane; l < L; l += 32) hits += line_f64_lean_inl(x, r64, -1, lines64[l], acc) ? 1 : 0;
    } else {
        // second pass: find this lane's flagged lines again (same float32 test) and redo them in float64
        const float4 q0 = r32[nf32::G1], q1 = r32[nf32::G2], q2 = r32[nf32::G3];
        const V3<float> g1 = mk(q0.x, q0.y, q0.z), g2 = mk(q1.x, q1.y, q1.z), g3 = mk(q2.x, q2.y, q2.z);
        const V3<float> g0 = mk(-(g1.x + g2.x + g3.x), -(g1.y + g2.y + g3.y), -(g1.z + g2.z + g3.z));
        const float4 ch = r32[nf32::CH], cm = r32[nf32::CM];
        const V3<float> rc = mk((ch.x - xh0) + (cm.x - xm0), (ch.y - xh1) + (cm.y - xm1), (ch.z - xh2) + (cm.z - xm2));
        const float rc2 = dot3(rc, rc), bound = q1.w * (1.0f + kBoundPadF);
        const float f = kVertexFallback * kVertexFallback;
#pragma unroll 1
        for (int l = lane; l < L; l += 32) {
            const float4 ln = lines[l];
            const V3<float> s = mk(ln.x, ln.y, ln.z);
            const float rs = dot3(rc, s);
            if (rc2 - rs * rs > bound) continue;
            const float b1 = dot3(g1, s), b2 = dot3(g2, s), b3 = dot3(g3, s), b0 = -(b1 + b2 + b3);
            const bool redo = (vk != 0 && b0 * b0 <= f * dot3(g0, g0)) || (vk != 1 && b1 * b1 <= f * dot3(g1, g1)) ||
                              (vk != 2 && b2 * b2 <= f * dot3(g2, g2)) || (vk != 3 && b3 * b3 <= f * dot3(g3, g3));
            if (redo && line_f64_lean_inl(x, r64, vk, lines64[l], acc)) ++hits;
        }
    }
}

// ---------------------------------------------------------------------------
// The velocity kernel.
// ---------------------------------------------------------------------------

// Bump allocator over the dynamic shared memory; every region starts on a 16-byte boundary.
struct SmemCarve {
    unsigned char *p;
    __device__ unsigned char *take(size_t bytes)
    {
        unsigned char *r = p;
        p += (bytes + 15) & ~(size_t)15;
        return r;
    }
};
__host__ __device__ constexpr size_t round16(size_t b) { return (b + 15) & ~(size_t)15; }

template <int S>
struct Pipe {
    uint64_t full[S];  // bulk copy of the tile in stage s has landed
    int done[S];       // warps finished with stage s (the last one refills it)
};

// Points: the block holds BP = NT*P consecutive points of the spatial order;
// warp w owns the 32*P consecutive slots [w*32*P, (w+1)*32*P), lane l the
// slots w*32*P + p*32 + l.  A warp therefore covers a compact patch of
// points, and a tile whose tets are all far from that patch skips the
// per-pair near/far test (culled=true below).
// The near pairs of a warp's queue, 32 at a time over the lanes: round r gives lane i the (32 r + i)-th
// pair in queue order (entry e, the k-th set lane of its mask).  (e0, k0) is the round's first pair.
struct PairCursor {
    int e0 = 0, k0 = 0;
};
// This lane's pair of the round: its entry and the point lane it belongs to (false past the last pair).
__device__ __forceinline__ bool cursor_pair(const PairCursor &c, const uint32_t *wm, int qn, int lane, int &e,
                                            int &owner)
{
    e = c.e0;
    int k = c.k0 + lane;
    while (e < qn && k >= __popc(wm[e])) {
        k -= __popc(wm[e]);
        ++e;
    }
    if (e >= qn) return false;
    unsigned m = wm[e];
    for (int i = 0; i < k; ++i) m &= m - 1u;
    owner = __ffs(m) - 1;
    return true;
}
__device__ __forceinline__ void cursor_advance(PairCursor &c, const uint32_t *wm, int qn)
{
    int k = c.k0 + 32;
    while (c.e0 < qn && k >= __popc(wm[c.e0])) {
        k -= __popc(wm[c.e0]);
        ++c.e0;
    }
    c.k0 = k;
}

// EXACT: near pairs take the exact integral (tet_exact) instead of the ray rule, the
// warp's pairs spread over all 32 lanes and each result handed to the lane that owns its point.
// DR: the near-pair drain's routine is called (0), inlined (1), or inlined in its lean form with the
// pair's state in the warp's shared slot (2); or (3) there is no drain: the near pairs are left out of
// the sums and counted, and the near pass (near_pass_kernel) evaluates them.  U: lines per lane per iteration of the ray rule (the ray bundle).
// UJ: the float32 far sweep's tet loop unrolled by UJ (two tets' chains interleave).
// PK (float32): the far sweep's packed f32x2 registers pair two evaluation points of the thread
// (the far record holds every value twice: the point-pair layout) instead of two quadrature points.
template <typename T, int Q, int P, int NT, int TILE, int S, int MINB, int DR, bool EXACT, int U, bool PK, int UJ>
__global__ void __launch_bounds__(NT, MINB) velocity_kernel(const VelocityArgs a)
{
    static_assert(!PK || (sizeof(T) == 4 && P % 2 == 0), "the point-pair sweep is float32 with an even P");
    constexpr int RS = far_stride<T>(Q, PK ? kFarPointPairs : kFarQuadPairs);
    constexpr int BP = NT * P;
    constexpr int NW = NT / 32;
    constexpr int QCAP = P * TILE;  // one entry per (tet, point row) of the tile: drained between tiles only
    constexpr int TILE_BYTES = TILE * RS * (int)sizeof(T);
    constexpr int HDR_BYTES = 32;  // tile header (two float4) in front of each stage's records
    constexpr int STAGE_BYTES = HDR_BYTES + TILE_BYTES;
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int NACC = F32 ? 6 : 3;  // float: (sum, compensation) per component; double: sum
    static_assert(TILE <= 256, "tet index in the near queue is 8 bits");

    if (a.skip && *a.skip) return;  // the mesh walk evaluated these points
    extern __shared__ __align__(128) unsigned char smem[];
    // shared-memory regions, each rounded up to 16 bytes (the same rule as smem_bytes below)
    SmemCarve carve{smem};
    unsigned char *stages = carve.take(S * STAGE_BYTES);                              // [S][header + TILE*RS]
    float *spts = reinterpret_cast<float *>(carve.take(9 * sizeof(float) * BP));      // [BP][3][hi, mid, lo]
    // near queue per warp: (lane mask, point row p << 8 | tet j) for each (j, p) with a near pair
    uint32_t *qmask = reinterpret_cast<uint32_t *>(carve.take(sizeof(uint32_t) * NW * QCAP));  // [NW][QCAP]
    uint16_t *qcode = reinterpret_cast<uint16_t *>(carve.take(sizeof(uint16_t) * NW * QCAP));  // [NW][QCAP]
    float4 *srec = reinterpret_cast<float4 *>(carve.take(sizeof(float4) * NW * kNearF32Vec4));  // staged near records
    Pipe<S> *pipe = reinterpret_cast<Pipe<S> *>(carve.take(sizeof(Pipe<S>)));
    MeshDesc *s_md = reinterpret_cast<MeshDesc *>(carve.take(sizeof(MeshDesc)));
    int64_t *s_item = reinterpret_cast<int64_t *>(carve.take(16));
    // per-point state, touched once per tile: compensated sums [NACC][BP] and counts [2][BP]
    // (near pairs, chord hits); the warp's bounding sphere [NW]
    T *sacc = reinterpret_cast<T *>(carve.take(sizeof(T) * NACC * BP));
    int *scnt = reinterpret_cast<int *>(carve.take(sizeof(int) * 2 * BP));
    float4 *swarp = reinterpret_cast<float4 *>(carve.take(sizeof(float4) * NW));
    float4 *sslot = reinterpret_cast<float4 *>(carve.take(sizeof(float4) * NW * kPairSlotVec4));  // lean drain
    uint32_t *sredo = reinterpret_cast<uint32_t *>(carve.take(sizeof(uint32_t) * NW * 32));      // its float64 redo list
    // direction table last: its size depends on the launch, every region above has a fixed offset
    float4 *sdir = reinterpret_cast<float4 *>(carve.take(a.smem_lines ? sizeof(float4) * a.L : 0));
    if (F32 && a.smem_lines)
        for (int l = threadIdx.x; l < a.L; l += NT) sdir[l] = a.lines.f32[l];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // far ratio squared in T, and the far ratio in float (+inf for the all-ray rule): kernel parameters
    // read where they are used, not held in registers across the loops
    auto fr2 = [&]() -> T {
        if constexpr (F32) return a.far_ratio2_f;
        else return a.far_ratio2;
    };
    const MeshDesc &md = *s_md;  // mesh of the current item (shared memory)

    if (tid == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&pipe->full[st], 1);
            pipe->done[st] = 0;
        }
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0u;  // bit st: parity of the next completion of full[st]

    auto issue = [&](int t, int st) {
        const int64_t first = (int64_t)t * TILE;
        const int cnt = (int)min((int64_t)TILE, md.n_tets - first);
        const uint32_t bytes = (uint32_t)cnt * RS * sizeof(T);
        unsigned char *dst = stages + st * STAGE_BYTES;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&pipe->full[st], bytes + HDR_BYTES);
        if (a.withhold_copies) return;
        bulk_g2s(dst, md.tile_hdr + 2 * t, HDR_BYTES, &pipe->full[st]);
        bulk_g2s(dst + HDR_BYTES, reinterpret_cast<const T *>(md.far) + first * RS, bytes, &pipe->full[st]);
    };
    auto wait_cap = [&]() -> long long { return a.wait_polls > 0 ? a.wait_polls : kWaitCap; };

    for (;;) {
        if (tid == 0) {
            int64_t item = atomicAdd(a.work_counter, 1ull);
            if (item < a.n_items) {
                if (a.meshes) {
                    // the mesh whose item range holds this item (binary search on item_begin)
                    int lo = 0, hi = a.n_meshes - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (a.meshes[mid].item_begin <= item) lo = mid;
                        else hi = mid - 1;
                    }
                    *s_md = a.meshes[lo];
                    item -= s_md->item_begin;
                } else {
                    *s_md = a.m;
                }
            } else {
                item = -1;
            }
            *s_item = item;
        }
        __syncthreads();
        // 32-bit item arithmetic: points, tiles and work items of a launch are below 2^31 (the host checks)
        const int item = (int)*s_item;
        if (item < 0) break;
        const int k = (int)md.k;
        const int n_blocks = (k + BP - 1) / BP;
        const int n_tiles = (int)((md.n_tets + TILE - 1) / TILE);
        const int pb = item % n_blocks, ck = item / n_blocks;
        const int t0 = ck * md.tiles_per_chunk;
        const int t1 = min(t0 + md.tiles_per_chunk, n_tiles);
        const int n_local = t1 - t0;

        // prologue: fill every stage while the points are loaded
        if (tid == 0)
            for (int i = 0; i < S && i < n_local; ++i) issue(t0 + i, i);

        for (int i = tid; i < BP; i += NT) {
            int gi = pb * BP + i;
            if (gi >= k) gi = k - 1;  // pad with a real point; its result is not written
            const int64_t src = md.perm[gi];
#pragma unroll
            for (int j = 0; j < 3; ++j) split3(md.pts[3 * src + j], spts[9 * i + 3 * j], spts[9 * i + 3 * j + 1],
                                               spts[9 * i + 3 * j + 2]);
        }
        __syncthreads();

        const int slot0 = warp * 32 * P + lane;  // block slot of this thread's point p: slot0 + 32 p
#pragma unroll
        for (int p = 0; p < P; ++p) {
#pragma unroll
            for (int j = 0; j < NACC; ++j) sacc[j * BP + slot0 + 32 * p] = 0;
            scnt[slot0 + 32 * p] = 0;
            scnt[BP + slot0 + 32 * p] = 0;
        }
        // bounding sphere of the warp's points (float, padded)
        {
            float mnx = INFINITY, mxx = -INFINITY, mny = INFINITY, mxy = -INFINITY, mnz = INFINITY, mxz = -INFINITY;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float *sp = spts + 9 * (slot0 + 32 * p);
                mnx = fminf(mnx, sp[0]); mxx = fmaxf(mxx, sp[0]);
                mny = fminf(mny, sp[3]); mxy = fmaxf(mxy, sp[3]);
                mnz = fminf(mnz, sp[6]); mxz = fmaxf(mxz, sp[6]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
                mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
                mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
                mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
                mnz = fminf(mnz, __shfl_xor_sync(0xffffffffu, mnz, o));
                mxz = fmaxf(mxz, __shfl_xor_sync(0xffffffffu, mxz, o));
            }
            const float ex = mxx - mnx, ey = mxy - mny, ez = mxz - mnz;
            if (lane == 0)
                swarp[warp] = make_float4(0.5f * (mnx + mxx), 0.5f * (mny + mxy), 0.5f * (mnz + mxz),
                                          0.5f * sqrtf(ex * ex + ey * ey + ez * ez) * 1.001f + 1e-6f);
            __syncwarp();
        }
        uint32_t *wm = qmask + warp * QCAP;
        uint16_t *wc = qcode + warp * QCAP;

        bool aborted = false;
#pragma unroll 1
        for (int i = 0; i < n_local; ++i) {
            const int st = i % S;
            const int t = t0 + i;
            // the warp gives up as one (a lane that saw the copy land leaves with the others)
            if (!__all_sync(0xffffffffu, mbar_wait(&pipe->full[st], (phase >> st) & 1u, wait_cap()))) {
                aborted = true;
                break;
            }
            phase ^= 1u << st;
            const float4 *sh = reinterpret_cast<const float4 *>(stages + st * STAGE_BYTES);
            const float4 hd = sh[0];
            const T *tb = reinterpret_cast<const T *>(stages + st * STAGE_BYTES + HDR_BYTES);
            // can any point of this warp be near a tet of this tile?
            const bool culled = !a.all_ray && tile_culled(swarp[warp], hd, sh[1].x, a.far_ratio_f);
            const int cnt = (int)min((int64_t)TILE, md.n_tets - (int64_t)t * TILE);
            int qn = 0;  // warp-uniform
            // this warp is done with stage st (the near pairs read global memory only);
            // the last warp to finish refills it
            auto release = [&]() {
                __syncwarp();
                if (lane == 0) {
                    __threadfence_block();
                    const int prev = atomicAdd(&pipe->done[st], 1);
                    if (prev == NW - 1) {
                        pipe->done[st] = 0;
                        __threadfence_block();
                        if (i + S < n_local) issue(t + S, st);
                    }
                }
            };

            if constexpr (F32) {
                // tile frame: x' = x - o.  Quadrature-pair sweep (PK = false): the two halves of a packed
                // f32x2 register are two quadrature points of the same evaluation point; point-pair sweep
                // (PK): two evaluation points of this thread against the same quadrature point.
                constexpr int NR = PK ? P / 2 : P;               // packed register sets
                constexpr int NQ = PK ? Q : (Q + 1) / 2;          // record groups of five float4 per tet
                float xs_[P][3];                                  // x' of each point (classification, x' x A)
                unsigned long long x2[NR][3], xx2[NR], A2[NR][3], B2[NR][3];
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float *sp = spts + 9 * (slot0 + 32 * p);
                    xs_[p][0] = sp[0] - hd.x;
                    xs_[p][1] = sp[3] - hd.y;
                    xs_[p][2] = sp[6] - hd.z;
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int pa = PK ? 2 * r : r, pb = PK ? 2 * r + 1 : r;
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj) x2[r][jj] = pack2(xs_[pa][jj], xs_[pb][jj]);
                    const float xxa = xs_[pa][0] * xs_[pa][0] + xs_[pa][1] * xs_[pa][1] + xs_[pa][2] * xs_[pa][2];
                    const float xxb = xs_[pb][0] * xs_[pb][0] + xs_[pb][1] * xs_[pb][1] + xs_[pb][2] * xs_[pb][2];
                    xx2[r] = pack2(xxa, xxb);
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj) A2[r][jj] = B2[r][jj] = 0ull;
                }
                // x' of point p (read back from the packed registers, which keep it live once)
                auto xl = [&](int p, int jj) {
                    float lo, hi;
                    unpack2(x2[PK ? p / 2 : p][jj], lo, hi);
                    return (PK && (p & 1)) ? hi : lo;
                };
                const float4 *tb4 = reinterpret_cast<const float4 *>(tb);
                // far sweep over the tile; MIXED: per-pair near/far test, near pairs masked and queued
                auto sweep = [&](auto mixed_tag) {
                    constexpr bool MIXED = decltype(mixed_tag)::value;
#pragma unroll UJ
                    for (int j = 0; j < cnt; ++j) {
                        const float4 *rec = tb4 + j * (RS / 4);
                        const ulonglong2 *rec2 = reinterpret_cast<const ulonglong2 *>(rec);
                        bool nearp[P];
                        if constexpr (MIXED) {
                            const float4 h0 = rec[0];
#pragma unroll
                            for (int p = 0; p < P; ++p) nearp[p] = pair_is_near_f32(xl(p, 0), xl(p, 1), xl(p, 2), h0, fr2());
                        }
#pragma unroll
                        for (int g = 0; g < NQ; ++g) {
                            // (mx, my) (mz, qq) (wx, wy) (wz, bx) (by, bz), each a packed pair: of two
                            // quadrature points, or (PK) one quadrature point's value twice
                            const ulonglong2 v0 = rec2[1 + 5 * g], v1 = rec2[2 + 5 * g], v2 = rec2[3 + 5 * g],
                                             v3 = rec2[4 + 5 * g], v4 = rec2[5 + 5 * g];
#pragma unroll
                            for (int r = 0; r < NR; ++r) {
                                const unsigned long long r2 =
                                    fma2(x2[r][0], v0.x, fma2(x2[r][1], v0.y, fma2(x2[r][2], v1.x, add2(xx2[r], v1.y))));
                                float ra, rb;
                                unpack2(r2, ra, rb);
                                float ia = rsqrt_ftz(ra), ib = rsqrt_ftz(rb);
                                if constexpr (MIXED && PK) {
                                    ia = nearp[2 * r] ? 0.f : ia;
                                    ib = nearp[2 * r + 1] ? 0.f : ib;
                                }
                                const unsigned long long ir = pack2(ia, ib);
                                unsigned long long ir3 = mul2(mul2(ir, ir), ir);
                                if constexpr (MIXED && !PK) ir3 = nearp[r] ? 0ull : ir3;
                                A2[r][0] = fma2(ir3, v2.x, A2[r][0]);
                                A2[r][1] = fma2(ir3, v2.y, A2[r][1]);
                                A2[r][2] = fma2(ir3, v3.x, A2[r][2]);
                                B2[r][0] = fma2(ir3, v3.y, B2[r][0]);
                                B2[r][1] = fma2(ir3, v4.x, B2[r][1]);
                                B2[r][2] = fma2(ir3, v4.y, B2[r][2]);
                            }
                        }
                        if constexpr (MIXED && DR == 3) {  // counted here, evaluated by the near pass
#pragma unroll
                            for (int p = 0; p < P; ++p)
                                if (nearp[p]) ++scnt[slot0 + 32 * p];
                        } else if constexpr (MIXED) {
#pragma unroll
                            for (int p = 0; p < P; ++p) {
                                const unsigned m = __ballot_sync(0xffffffffu, nearp[p]);
                                if (m) {
                                    if (lane == 0) {
                                        wm[qn] = m;
                                        wc[qn] = (uint16_t)((p << 8) | j);
                                    }
                                    if (nearp[p]) ++scnt[slot0 + 32 * p];
                                    ++qn;
                                }
                            }
                        }
                    }
                };
                if (culled)
                    sweep(std::false_type{});
                else
                    sweep(std::true_type{});
                float A[P][3], B[P][3];
#pragma unroll
                for (int r = 0; r < NR; ++r)
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj) {
                        if constexpr (PK) {
                            unpack2(A2[r][jj], A[2 * r][jj], A[2 * r + 1][jj]);
                            unpack2(B2[r][jj], B[2 * r][jj], B[2 * r + 1][jj]);
                        } else {
                            A[r][jj] = sum2(A2[r][jj]);
                            B[r][jj] = sum2(B2[r][jj]);
                        }
                    }
                release();
                // compensated add of v into the sums of block slot sl
                auto kahan = [&](int sl, float v0, float v1, float v2) {
                    const float v[3] = {v0, v1, v2};
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj) {
                        float &sum = sacc[(2 * jj) * BP + sl];
                        float &cmp = sacc[(2 * jj + 1) * BP + sl];
                        const float y = v[jj] - cmp;
                        const float s2 = sum + y;
                        cmp = (s2 - sum) - y;
                        sum = s2;
                    }
                };
                // far part of the tile: x' x A - B
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float x = xl(p, 0), y = xl(p, 1), z = xl(p, 2);
                    kahan(slot0 + 32 * p, y * A[p][2] - z * A[p][1] - B[p][0], z * A[p][0] - x * A[p][2] - B[p][1],
                          x * A[p][1] - y * A[p][0] - B[p][2]);
                }
                // near pairs of the tile: the warp takes them one at a time; each tet's near record is
                // staged once (one coalesced load into this warp's shared slot, read by broadcast)
                if (EXACT && qn > 0) {
                    __syncwarp();
                    PairCursor cur;
#pragma unroll 1
                    while (cur.e0 < qn) {
                        int e = 0, owner = 0, tag = 0;
                        float ox = 0.f, oy = 0.f, oz = 0.f;
                        if (cursor_pair(cur, wm, qn, lane, e, owner)) {
                            const int code = wc[e];
                            const int pp = code >> 8, j = code & 255;
                            const float *sp = spts + 9 * (warp * 32 * P + pp * 32 + owner);
                            const V3<double> xd = mk(join3(sp[0], sp[1], sp[2]), join3(sp[3], sp[4], sp[5]),
                                                     join3(sp[6], sp[7], sp[8]));
                            const Vel64 o = tet_exact<true>(xd, md.near64 + ((int64_t)t * TILE + j) * kNearF64);
                            ox = (float)o.x;
                            oy = (float)o.y;
                            oz = (float)o.z;
                            tag = 1 | (pp << 1) | (owner << 8);
                        }
                        cursor_advance(cur, wm, qn);
#pragma unroll 1
                        for (int src = 0; src < 32; ++src) {
                            const int tg = __shfl_sync(0xffffffffu, tag, src);
                            const float sx = __shfl_sync(0xffffffffu, ox, src);
                            const float sy = __shfl_sync(0xffffffffu, oy, src);
                            const float sz = __shfl_sync(0xffffffffu, oz, src);
                            if ((tg & 1) && (tg >> 8) == lane) kahan(warp * 32 * P + ((tg >> 1) & 127) * 32 + lane, sx, sy, sz);
                        }
                    }
                    __syncwarp();
                } else if (DR != 3 && qn > 0) {
                    __syncwarp();
                    int held = -1;
#pragma unroll 1
                    for (int e = 0; e < qn; ++e) {
                        unsigned m = wm[e];
                        const int code = wc[e];
                        const int pp = code >> 8, j = code & 255;
                        const int64_t tet = (int64_t)t * TILE + j;
                        if (j != held) {
                            __syncwarp();
                            if (lane < kNearF32Vec4)
                                srec[warp * kNearF32Vec4 + lane] = md.near32[tet * kNearF32Vec4 + lane];
                            __syncwarp();
                            held = j;
                        }
                        int n_redo = 0;  // lean drain: pairs of this entry queued for their float64 steps
#pragma unroll 1
                        while (m) {
                            const int owner = __ffs(m) - 1;
                            m &= m - 1u;
                            const int bi = warp * 32 * P + pp * 32 + owner;
                            NearOut32 o;
                            if constexpr (DR == 2) {
                                bool redo = false, whole = false;
                                int vk = -1;
                                o = near_pair_f32_lean<U>(spts + 9 * bi, srec + warp * kNearF32Vec4,
                                                          a.smem_lines ? sdir : a.lines.f32, a.L, lane,
                                                          sslot + warp * kPairSlotVec4, &redo, &vk, &whole);
                                if (redo) {  // warp-uniform
                                    if (lane == 0)
                                        sredo[warp * 32 + n_redo] = (uint32_t)bi | ((uint32_t)(vk + 1) << 16) |
                                                                    (whole ? 1u << 20 : 0u);
                                    ++n_redo;
                                }
                            } else if constexpr (DR == 1)
                                o = near_pair_f32_body<U>(spts + 9 * bi, srec + warp * kNearF32Vec4,
                                                          md.near64 + tet * kNearF64, a.smem_lines ? sdir : a.lines.f32,
                                                          a.lines.f64, a.L, lane);
                            else
                                o = near_pair_f32<U>(spts + 9 * bi, srec + warp * kNearF32Vec4,
                                                     md.near64 + tet * kNearF64, a.smem_lines ? sdir : a.lines.f32,
                                                     a.lines.f64, a.L, lane);
                            if (lane == owner) {
                                kahan(bi, o.vx, o.vy, o.vz);
                                scnt[BP + bi] += o.hits;
                            }
                        }
                        if constexpr (DR == 2) {
                            // the float64 steps of the entry's flagged pairs (at most one per lane of the mask)
                            __syncwarp();
#pragma unroll 1
                            for (int f = 0; f < n_redo; ++f) {
                                const uint32_t c = sredo[warp * 32 + f];
                                const int bi = (int)(c & 0xffffu), vk = (int)((c >> 16) & 15u) - 1;
                                const bool whole = (c >> 20) & 1u;
                                const float *xs = spts + 9 * bi;
                                const V3<double> x = mk(join3(xs[0], xs[1], xs[2]), join3(xs[3], xs[4], xs[5]),
                                                        join3(xs[6], xs[7], xs[8]));
                                V3<double> acc = mk(0.0, 0.0, 0.0);
                                int hits = 0;
                                line_fallback_f64_inl(x, xs, srec + warp * kNearF32Vec4, md.near64 + tet * kNearF64,
                                                      a.smem_lines ? sdir : a.lines.f32, a.lines.f64, a.L, lane, vk,
                                                      whole, acc, hits);
                                const double vx = warp_sum(acc.x), vy = warp_sum(acc.y), vz = warp_sum(acc.z);
                                hits = warp_sum(hits);
                                if (lane == (bi & 31)) {
                                    kahan(bi, (float)vx, (float)vy, (float)vz);
                                    scnt[BP + bi] += hits;
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
            } else {
                // float64: near/far test in global coordinates, far rule in the tile frame
                double tacc[P][3];
                V3<double> xp[P];
                // tile frame x' = x - o (exact: the origin is a float), as in the float32 sweep
                V3<double> xl[P];
                double xx[P], A[P][3], B[P][3];
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    tacc[p][0] = tacc[p][1] = tacc[p][2] = 0.0;
                    const float *sp = spts + 9 * (slot0 + 32 * p);
                    xp[p] = mk(join3(sp[0], sp[1], sp[2]), join3(sp[3], sp[4], sp[5]), join3(sp[6], sp[7], sp[8]));
                    xl[p] = mk(xp[p].x - (double)hd.x, xp[p].y - (double)hd.y, xp[p].z - (double)hd.z);
                    xx[p] = xl[p].x * xl[p].x + xl[p].y * xl[p].y + xl[p].z * xl[p].z;
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj) A[p][jj] = B[p][jj] = 0.0;
                }
#pragma unroll 1
                for (int j = 0; j < cnt; ++j) {
                    const double *rec = tb + j * RS;
                    bool nearp[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) nearp[p] = !culled && pair_is_near_f64(xp[p].x, xp[p].y, xp[p].z, rec, fr2());
                    // per point q: (-2 x_q', |x_q'|^2, w', B = x_q' x w'); sum (x' - x_q') x w' / r^3 = x' x A - B
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        const double *qq = rec + 4 + 10 * q;
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            if (nearp[p]) continue;
                            const double r2 = fma(xl[p].x, qq[0], fma(xl[p].y, qq[1], fma(xl[p].z, qq[2], xx[p] + qq[3])));
                            const double ir = rsqrt(r2);  // one library call instead of a sqrt and a divide
                            const double ir3 = ir * ir * ir;
                            A[p][0] = fma(ir3, qq[4], A[p][0]);
                            A[p][1] = fma(ir3, qq[5], A[p][1]);
                            A[p][2] = fma(ir3, qq[6], A[p][2]);
                            B[p][0] = fma(ir3, qq[7], B[p][0]);
                            B[p][1] = fma(ir3, qq[8], B[p][1]);
                            B[p][2] = fma(ir3, qq[9], B[p][2]);
                        }
                    }
                    if (!culled && DR == 3) {
#pragma unroll
                        for (int p = 0; p < P; ++p)
                            if (nearp[p]) ++scnt[slot0 + 32 * p];
                    } else if (!culled) {
#pragma unroll
                        for (int p = 0; p < P; ++p) {
                            const unsigned m = __ballot_sync(0xffffffffu, nearp[p]);
                            if (m) {
                                if (lane == 0) {
                                    wm[qn] = m;
                                    wc[qn] = (uint16_t)((p << 8) | j);
                                }
                                if (nearp[p]) ++scnt[slot0 + 32 * p];
                                ++qn;
                            }
                        }
                    }
                }
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    tacc[p][0] += xl[p].y * A[p][2] - xl[p].z * A[p][1] - B[p][0];
                    tacc[p][1] += xl[p].z * A[p][0] - xl[p].x * A[p][2] - B[p][1];
                    tacc[p][2] += xl[p].x * A[p][1] - xl[p].y * A[p][0] - B[p][2];
                }
                release();
                if (EXACT && qn > 0) {
                    __syncwarp();
                    PairCursor cur;
#pragma unroll 1
                    while (cur.e0 < qn) {
                        int e = 0, owner = 0, tag = 0;
                        Vel64 o = {0.0, 0.0, 0.0};
                        if (cursor_pair(cur, wm, qn, lane, e, owner)) {
                            const int code = wc[e];
                            const int pp = code >> 8, j = code & 255;
                            const float *sp = spts + 9 * (warp * 32 * P + pp * 32 + owner);
                            const V3<double> xd = mk(join3(sp[0], sp[1], sp[2]), join3(sp[3], sp[4], sp[5]),
                                                     join3(sp[6], sp[7], sp[8]));
                            o = tet_exact<false>(xd, md.near64 + ((int64_t)t * TILE + j) * kNearF64);
                            tag = 1 | (pp << 1) | (owner << 8);
                        }
                        cursor_advance(cur, wm, qn);
#pragma unroll 1
                        for (int src = 0; src < 32; ++src) {
                            const int tg = __shfl_sync(0xffffffffu, tag, src);
                            const double sx = __shfl_sync(0xffffffffu, o.x, src);
                            const double sy = __shfl_sync(0xffffffffu, o.y, src);
                            const double sz = __shfl_sync(0xffffffffu, o.z, src);
                            if ((tg & 1) && (tg >> 8) == lane) {
                                const int pp = (tg >> 1) & 127;
#pragma unroll
                                for (int p = 0; p < P; ++p)
                                    if (p == pp) {
                                        tacc[p][0] += sx;
                                        tacc[p][1] += sy;
                                        tacc[p][2] += sz;
                                    }
                            }
                        }
                    }
                    __syncwarp();
                } else if (DR != 3 && qn > 0) {
                    __syncwarp();
#pragma unroll 1
                    for (int e = 0; e < qn; ++e) {
                        unsigned m = wm[e];
                        const int code = wc[e];
                        const int pp = code >> 8, j = code & 255;
                        const int64_t tet = (int64_t)t * TILE + j;
#pragma unroll 1
                        while (m) {
                            const int owner = __ffs(m) - 1;
                            m &= m - 1u;
                            const int bi = warp * 32 * P + pp * 32 + owner;
                            const float *sp = spts + 9 * bi;
                            const V3<double> xd = mk(join3(sp[0], sp[1], sp[2]), join3(sp[3], sp[4], sp[5]),
                                                     join3(sp[6], sp[7], sp[8]));
                            const NearOut o = near_pair_f64(xd, md.near64 + tet * kNearF64, a.lines.f64, a.L, lane);
                            if (lane == owner) {
#pragma unroll
                                for (int p = 0; p < P; ++p)
                                    if (p == pp) {
                                        tacc[p][0] += o.vx;
                                        tacc[p][1] += o.vy;
                                        tacc[p][2] += o.vz;
                                    }
                                scnt[BP + bi] += o.hits;
                            }
                        }
                    }
                    __syncwarp();
                }
#pragma unroll
                for (int p = 0; p < P; ++p)
#pragma unroll
                    for (int jj = 0; jj < 3; ++jj) sacc[jj * BP + slot0 + 32 * p] += tacc[p][jj];
            }
        }
        if (aborted) {
            if (tid == 0) atomicOr(a.flag, kFlagTimeout);
            mbar_drain<S>(pipe->full, phase, wait_cap());
            return;
        }

        const int64_t ntets_chunk = min(md.n_tets, (int64_t)t1 * TILE) - (int64_t)t0 * TILE;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int gi = pb * BP + warp * 32 * P + p * 32 + lane;  // position in the spatial order
            if (gi >= k) continue;
            double *dst = md.partial + ((int64_t)ck * k + gi) * 3;
            const int sl = slot0 + 32 * p;
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
                if constexpr (F32)
                    dst[jj] = (double)sacc[(2 * jj) * BP + sl] - (double)sacc[(2 * jj + 1) * BP + sl];
                else
                    dst[jj] = sacc[jj * BP + sl];
            }
            if (a.counts) {
                const int64_t src = md.perm[gi];
                const int nnear = scnt[sl];
                atomicAdd(&a.counts[3 * src + 0], nnear);
                atomicAdd(&a.counts[3 * src + 1], (int)(ntets_chunk - nnear));
                atomicAdd(&a.counts[3 * src + 2], scnt[BP + sl]);
            }
        }
        __syncthreads();  // stages and points are reused by the next item
    }
}

template <typename T, int Q, int P, int NT, int TILE, int S, bool PK>
size_t smem_bytes(int lines_in_smem)
{
    constexpr int RS = far_stride<T>(Q, PK ? kFarPointPairs : kFarQuadPairs);
    constexpr size_t NW = NT / 32;
    return round16((size_t)S * (32 + TILE * RS * sizeof(T))) + round16(9 * sizeof(float) * NT * P) +
           round16(sizeof(uint32_t) * NW * P * TILE) + round16(sizeof(uint16_t) * NW * P * TILE) +
           round16(sizeof(float4) * NW * kNearF32Vec4) + round16(sizeof(Pipe<S>)) +
           round16(sizeof(MeshDesc)) + 16 + round16(sizeof(float4) * lines_in_smem) +
           round16(sizeof(T) * (sizeof(T) == 4 ? 6 : 3) * NT * P) + round16(sizeof(int) * 2 * NT * P) +
           round16(sizeof(float4) * NW) + round16(sizeof(float4) * NW * kPairSlotVec4) +
           round16(sizeof(uint32_t) * NW * 32);
}

template <typename T, int Q, int P, int NT, int TILE, int S, int MINB, int DR, bool EXACT, int U, bool PK, int UJ>
cudaError_t launch_t(const VelocityArgs &a, int n_sm, cudaStream_t st, int *grid_out, bool query_only, int *occ_out)
{
    auto kern = velocity_kernel<T, Q, P, NT, TILE, S, MINB, DR, EXACT, U, PK, UJ>;
    const size_t sm = smem_bytes<T, Q, P, NT, TILE, S, PK>(a.smem_lines ? a.L : 0);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, sm);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (occ_out) *occ_out = occ;
    if (query_only) return cudaSuccess;
    const int64_t grid = std::min<int64_t>(a.n_items, (int64_t)n_sm * occ);
    if (grid_out) *grid_out = (int)grid;
    kern<<<(unsigned)grid, NT, sm, st>>>(a);
    return cudaGetLastError();
}


}  // namespace
}  // namespace bs
