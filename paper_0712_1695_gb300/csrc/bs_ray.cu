// bs_ray.cu -- the all-ray evaluation: the ray rule of Section 2 (Eq. 2-5) for every
// (point, tet) pair, far_ratio = +inf, the paper's own method (§2.2 step 4), as a kernel
// of its own.
//
// The velocity kernel (bs_velocity.cu) gives near pairs to the whole warp: the 32 lanes
// split the lines of one pair and reduce with shuffles, which suits the ~100 near tets of
// a node.  In the all-ray method every tet is near, so here one thread takes one point and
// walks the tets of the chunk itself, with no reduction: items are (block of 128 points in
// spatial order, chunk of consecutive tets), pulled from a device counter by a persistent
// grid; the chunk's near records stream through a two-stage shared-memory ring (one bulk
// copy per tile of 32 tets, mbarrier, the last warp to finish a stage refills it).
//
// Direction window.  A line x + t s can reach the tet only if it passes within Rb of the
// centroid c (the bounding-sphere test of the ray rule); with u the direction of c - x and
// sin(alpha) = Rb / |c - x|, that needs s within alpha of u or of -u, so its polar angle
// phi lies within alpha of phi(u) or of pi - phi(u).  The warp's 32 points lie in a small
// ball (they are consecutive in the spatial order), so one window, widened by the angle the
// ball subtends, serves the warp: its lanes take the same lines in lock step (broadcast
// reads of the direction table, no divergence between lanes' loops).  Only the phi-rings of
// the direction table (Eq. 3: l = n * n_theta + m, phi ascending in n) inside the window are
// visited, padded by more than the rounding of the float32 test; every visited line still
// takes each lane's exact bounding-sphere test, so the set of lines that contribute is the
// one of the dense loop over all n_phi * n_theta lines.  For a tet a few warp sizes away this
// visits a few rings instead of all of them.
//
// Per line the arithmetic is the velocity kernel's (barycentric clipping of the line,
// Eq. 5 with sign(t)); float64 steps for the same degenerate cases: x a vertex of the tet
// with the line nearly in a face through it, or x within 1e-5 (barycentric) of the tet's
// boundary.  float32: per-tile sums Kahan-compensated across tiles; float64: plain sums.
// Each item writes its partial to scratch[chunk][point]; the reduce kernel adds the chunks
// in a fixed order.
#include <math.h>

#include <algorithm>

#include "bs_internal.cuh"
#include "bs_near.cuh"

namespace bs {
namespace {

constexpr int kRayThreads = 128;  // one point per thread
constexpr int kRayTile = 32;      // tets per shared-memory stage
constexpr int kRayStages = 2;

template <typename T>
constexpr int ray_rec_bytes()
{
    return sizeof(T) == 4 ? (int)sizeof(float4) * kNearF32Vec4 : (int)sizeof(double) * kNearF64;
}

struct RayPipe {
    uint64_t full[kRayStages];  // bulk copy of the tile in stage s has landed
    int done[kRayStages];       // warps finished with stage s
};

// first ring n with z_n <= v (lower) or z_n < v (upper); z_n = cos(phi_n) descends with n
template <typename T>
__device__ inline int ring_bound(const T *z, int n, T v, bool upper)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (upper ? (z[mid] >= v) : (z[mid] > v)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Rings [a0, a1) and [b0, b1) (ascending, disjoint) holding every line that can pass the
// bounding-sphere test of a tet (centroid c, test radius^2 bound, R = sqrt(bound)) for any point
// of a ball (centre cw, radius rw; D = c - cw, d = |D|).  For a point x of the ball a passing line
// has its direction within alpha_x of +-u_x (u_x = (c - x)/|c - x|, sin alpha_x = R/|c - x|),
// and u_x is within beta of u = D/d (sin beta = rw/d, the largest angle the ball subtends from
// c); with |c - x| >= d - rw, every such line is within alpha + beta of +-u, sin alpha =
// R/(d - rw).  The angle is padded by 2e-3 + 1e-6 (d + rw)/R radians: the float32 test decides
// |rc|^2 - (rc.s)^2 <= bound with an absolute error of about 1.1e-6 |rc|^2, which admits lines at
// most min(1.05e-3, 5.5e-7 |rc|/R) radians outside the exact cone, and the pad also covers the
// rounding of the window and of the table's z_n.  The sine and cosine of the padded angle are
// bounded (the pad's sine by the pad, its cosine by 1 - pad^2/2), which can only widen the
// window.  The windows are intervals of z = cos(phi): [zlo, zhi] around u, [-zhi, -zlo] around -u.
template <typename T>
__device__ inline void ring_window(const T *z, int N, V3<T> D, T rw, T bound, int &a0, int &a1, int &b0, int &b1)
{
    a0 = 0;
    a1 = N;
    b0 = b1 = 0;
    const T d = sqrt(dot3(D, D)), R = sqrt(bound);
    if (!(d - rw > (T)1.01 * R)) return;  // the ball reaches the tet's bounding sphere: every ring
    const T s1 = R / (d - rw), s2 = rw / d;
    const T c1 = sqrt((T)1 - s1 * s1), c2 = sqrt((T)1 - s2 * s2);
    const T sab = s1 * c2 + c1 * s2, cab = c1 * c2 - s1 * s2;  // sin, cos of alpha + beta
    const T pad = (T)2e-3 + (T)1e-6 * (d + rw) / R;
    if (!(pad < (T)0.25) || !(cab > (T)0)) return;
    const T sA = min((T)1, sab + cab * pad);
    const T cA = cab * ((T)1 - (T)0.5 * pad * pad) - sab * pad;
    if (!(cA > (T)0)) return;
    const T uz = D.z / d, su = sqrt(D.x * D.x + D.y * D.y) / d;
    const T zhi = uz <= cA ? uz * cA + su * sA : (T)1;   // cos(max(phi_u - alpha', 0))
    const T zlo = uz >= -cA ? uz * cA - su * sA : (T)-1;  // cos(min(phi_u + alpha', pi))
    a0 = ring_bound(z, N, zhi, false);
    a1 = ring_bound(z, N, zlo, true);
    b0 = ring_bound(z, N, -zlo, false);
    b1 = ring_bound(z, N, -zhi, true);
    if (b0 < a1 && a0 < b1) {  // the two windows overlap: one range
        a0 = min(a0, b0);
        a1 = max(a1, b1);
        b0 = b1 = 0;
    } else if (b0 < a0) {  // keep rings ascending
        const int t0 = a0, t1 = a1;
        a0 = b0;
        a1 = b1;
        b0 = t0;
        b1 = t1;
    }
}

// float32 ray rule for one tet against the 32 points of a warp (one per lane).  The warp
// tests the window's lines in lock step, 32 at a time (broadcast reads of the direction
// table in shared memory), each lane keeping a mask of the lines its own point passes; the
// line-independent set-up then runs once for the warp, and each lane clips only its own
// passing lines.  xs: the lane's point as float splits [component][hi, mid, lo]; r32: the
// near record (shared memory); r64: its float64 copy (global, read only by the float64
// steps); [a0, a1), [b0, b1): the warp's rings.  Adds the pair's k s x J to (ax, ay, az).
// Returns true when some of this lane's lines need the float64 steps (x on a vertex with the line nearly in
// a face through it, or x within 1e-5 of the tet's boundary): ray_tet_redo_f64 does them afterwards.
__device__ __forceinline__ bool ray_tet_f32(const float *__restrict__ xs, const float4 *__restrict__ r32,
                                            const float4 *__restrict__ lines, int M, int a0, int a1, int b0, int b1,
                                            float &ax, float &ay, float &az, int &hits)
{
    const float xh0 = xs[0], xm0 = xs[1], xh1 = xs[3], xm1 = xs[4], xh2 = xs[6], xm2 = xs[7];
    const float4 ch = r32[nf32::CH], cm = r32[nf32::CM];
    const V3<float> rc = mk((ch.x - xh0) + (cm.x - xm0), (ch.y - xh1) + (cm.y - xm1), (ch.z - xh2) + (cm.z - xm2));
    const float rc2 = dot3(rc, rc);
    const float bound = r32[nf32::G2].w * (1.0f + kBoundPadF);
    // window position w -> line l: the rings [a0, a1) then [b0, b1), n_theta lines each
    const int nA = (a1 - a0) * M, nW = nA + (b1 - b0) * M;
    const int lA = a0 * M, lB = b0 * M - nA;

    bool ready = false;  // warp-uniform
    bool any_redo = false;
    int vk = -1;
    bool whole_f64 = false;
    // per lane: the point's barycentric coordinates, the parallel and vertex-fallback thresholds, W_a;
    // the tet's face gradients and vorticity stay in the staged record and are read per line
    float a[4], par2[4], fb2[4], tau_h = 0.f;
    V3<float> Wa = mk(0.f, 0.f, 0.f);
#pragma unroll 1
    for (int w0 = 0; w0 < nW; w0 += 32) {
        const int nw = min(32, nW - w0);
        uint32_t mine = 0u;  // lines of this group that this lane's point passes
#pragma unroll 4
        for (int i = 0; i < nw; ++i) {
            const int wi = w0 + i;
            const float4 ln = lines[wi < nA ? lA + wi : lB + wi];
            const float rs = rc.x * ln.x + rc.y * ln.y + rc.z * ln.z;
            if (!(rc2 - rs * rs > bound)) mine |= 1u << i;
        }
        if (!__any_sync(0xffffffffu, mine != 0u)) continue;
        if (!ready) {
            ready = true;
            const float *vh = reinterpret_cast<const float *>(r32 + nf32::VH);
            const float *vm = reinterpret_cast<const float *>(r32 + nf32::VM);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (vk < 0 && vh[3 * i] == xh0 && vm[3 * i] == xm0 && vh[3 * i + 1] == xh1 && vm[3 * i + 1] == xm1 &&
                    vh[3 * i + 2] == xh2 && vm[3 * i + 2] == xm2)
                    vk = i;
            const float4 q0 = r32[nf32::G1], q1 = r32[nf32::G2], q2 = r32[nf32::G3];
            V3<float> g[4];
            g[1] = mk(q0.x, q0.y, q0.z);
            g[2] = mk(q1.x, q1.y, q1.z);
            g[3] = mk(q2.x, q2.y, q2.z);
            g[0] = mk(-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z));
            if (vk >= 0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = (i == vk) ? 1.0f : 0.0f;
            } else {
                const V3<float> d0 =
                    mk((xh0 - vh[0]) + (xm0 - vm[0]), (xh1 - vh[1]) + (xm1 - vm[1]), (xh2 - vh[2]) + (xm2 - vm[2]));
                a[1] = dot3(g[1], d0);
                a[2] = dot3(g[2], d0);
                a[3] = dot3(g[3], d0);
                a[0] = 1.0f - a[1] - a[2] - a[3];
                const float amin = fminf(fminf(a[0], a[1]), fminf(a[2], a[3]));
                const float aabs = fminf(fminf(fabsf(a[0]), fabsf(a[1])), fminf(fabsf(a[2]), fabsf(a[3])));
                whole_f64 = amin > -kDegenA && aabs < kDegenA;
            }
            float wa[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 t = r32[nf32::W + i];
                wa[0] += a[i] * t.x;
                wa[1] += a[i] * t.y;
                wa[2] += a[i] * t.z;
                const float gg = dot3(g[i], g[i]);
                par2[i] = kParF * kParF * gg;
                fb2[i] = (vk >= 0 && i != vk) ? kVertexFallback * kVertexFallback * gg : -1.0f;
            }
            Wa = mk(wa[0], wa[1], wa[2]);
            tau_h = (float)kTau * q0.w;
        }
#pragma unroll 1
        while (mine) {
            const int i = __ffs(mine) - 1;
            mine &= mine - 1u;
            const int wi = w0 + i;
            const int l = wi < nA ? lA + wi : lB + wi;
            const float4 ln = lines[l];
            const V3<float> s = mk(ln.x, ln.y, ln.z);
            const float4 q0 = lds4(r32 + nf32::G1), q1 = lds4(r32 + nf32::G2), q2 = lds4(r32 + nf32::G3);
            float b[4];
            b[1] = q0.x * s.x + q0.y * s.y + q0.z * s.z;
            b[2] = q1.x * s.x + q1.y * s.y + q1.z * s.z;
            b[3] = q2.x * s.x + q2.y * s.y + q2.z * s.z;
            b[0] = -(b[1] + b[2] + b[3]);
            bool redo = whole_f64;
#pragma unroll
            for (int k = 0; k < 4; ++k) redo = redo || (b[k] * b[k] <= fb2[k]);
            if (redo) {  // rare: this line in float64, in the second pass below
                any_redo = true;
                continue;
            }
            float lo = -INFINITY, hi = INFINITY;
            bool empty = false;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (b[k] * b[k] <= par2[k]) empty = empty || (a[k] < -kParF);
                else if (b[k] > 0.f) lo = fmaxf(lo, -a[k] / b[k]);
                else hi = fminf(hi, -a[k] / b[k]);
            }
            if (empty || !(hi - lo > tau_h)) continue;
            float Wb[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 t = lds4(r32 + nf32::W + k);
                Wb[0] += b[k] * t.x;
                Wb[1] += b[k] * t.y;
                Wb[2] += b[k] * t.z;
            }
            const float f1 = fabsf(hi) - fabsf(lo);
            const float f2 = 0.5f * (hi * fabsf(hi) - lo * fabsf(lo));
            const V3<float> J = mk(f1 * Wa.x + f2 * Wb[0], f1 * Wa.y + f2 * Wb[1], f1 * Wa.z + f2 * Wb[2]);
            ax += ln.w * (s.y * J.z - s.z * J.y);
            ay += ln.w * (s.z * J.x - s.x * J.z);
            az += ln.w * (s.x * J.y - s.y * J.x);
            ++hits;
        }
    }
    return any_redo;
}

// The float64 steps of ray_tet_f32 for this lane's point and one tet: the same float32 tests pick the
// lines again (the window's lines that pass the bounding test and need float64), each is redone in
// float64 and added to (ax, ay, az).  Run after the tile's tets, where few registers are live.
__device__ __forceinline__ void ray_tet_redo_f64(const float *__restrict__ xs, const float4 *__restrict__ r32,
                                                 const double *__restrict__ r64, const float4 *__restrict__ lines,
                                                 const dbl4 *__restrict__ lines64, int M, int a0, int a1, int b0,
                                                 int b1, float &ax, float &ay, float &az, int &hits)
{
    const float xh0 = xs[0], xm0 = xs[1], xh1 = xs[3], xm1 = xs[4], xh2 = xs[6], xm2 = xs[7];
    const float4 ch = r32[nf32::CH], cm = r32[nf32::CM];
    const V3<float> rc = mk((ch.x - xh0) + (cm.x - xm0), (ch.y - xh1) + (cm.y - xm1), (ch.z - xh2) + (cm.z - xm2));
    const float rc2 = dot3(rc, rc);
    const float bound = r32[nf32::G2].w * (1.0f + kBoundPadF);
    const int nA = (a1 - a0) * M, nW = nA + (b1 - b0) * M;
    const int lA = a0 * M, lB = b0 * M - nA;
    const float *vh = reinterpret_cast<const float *>(r32 + nf32::VH);
    const float *vm = reinterpret_cast<const float *>(r32 + nf32::VM);
    int vk = -1;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (vk < 0 && vh[3 * i] == xh0 && vm[3 * i] == xm0 && vh[3 * i + 1] == xh1 && vm[3 * i + 1] == xm1 &&
            vh[3 * i + 2] == xh2 && vm[3 * i + 2] == xm2)
            vk = i;
    const float4 q0 = r32[nf32::G1], q1 = r32[nf32::G2], q2 = r32[nf32::G3];
    V3<float> g[4];
    g[1] = mk(q0.x, q0.y, q0.z);
    g[2] = mk(q1.x, q1.y, q1.z);
    g[3] = mk(q2.x, q2.y, q2.z);
    g[0] = mk(-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z));
    bool whole_f64 = false;
    if (vk < 0) {
        const V3<float> d0 = mk((xh0 - vh[0]) + (xm0 - vm[0]), (xh1 - vh[1]) + (xm1 - vm[1]), (xh2 - vh[2]) + (xm2 - vm[2]));
        float a[4];
        a[1] = dot3(g[1], d0);
        a[2] = dot3(g[2], d0);
        a[3] = dot3(g[3], d0);
        a[0] = 1.0f - a[1] - a[2] - a[3];
        const float amin = fminf(fminf(a[0], a[1]), fminf(a[2], a[3]));
        const float aabs = fminf(fminf(fabsf(a[0]), fabsf(a[1])), fminf(fabsf(a[2]), fabsf(a[3])));
        whole_f64 = amin > -kDegenA && aabs < kDegenA;
    }
    float fb2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        fb2[i] = (vk >= 0 && i != vk) ? kVertexFallback * kVertexFallback * dot3(g[i], g[i]) : -1.0f;
    const V3<double> xd = mk(join3(xs[0], xs[1], xs[2]), join3(xs[3], xs[4], xs[5]), join3(xs[6], xs[7], xs[8]));
    V3<double> acc = mk(0.0, 0.0, 0.0);
#pragma unroll 1
    for (int wi = 0; wi < nW; ++wi) {
        const int l = wi < nA ? lA + wi : lB + wi;
        const float4 ln = lines[l];
        const float rs = rc.x * ln.x + rc.y * ln.y + rc.z * ln.z;
        if (rc2 - rs * rs > bound) continue;
        const V3<float> s = mk(ln.x, ln.y, ln.z);
        bool redo = whole_f64;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float bk = dot3(g[k], s);
            redo = redo || (bk * bk <= fb2[k]);
        }
        if (redo && line_f64_lean_inl(xd, r64, whole_f64 ? -1 : vk, lines64[l], acc)) ++hits;
    }
    ax += (float)acc.x;
    ay += (float)acc.y;
    az += (float)acc.z;
}

// float64 form of ray_tet_f32 (the velocity kernel's line_f64 per line); r: the near record.
__device__ __forceinline__ void ray_tet_f64(V3<double> x, const double *__restrict__ r,
                                            const dbl4 *__restrict__ lines64, int M, int a0, int a1, int b0, int b1,
                                            V3<double> &acc, int &hits)
{
    const V3<double> rc = mk(r[nf64::C] - x.x, r[nf64::C + 1] - x.y, r[nf64::C + 2] - x.z);
    const double rc2 = dot3(rc, rc);
    const double bound = r[nf64::RB2] * (1.0 + kBoundPadD);
    PairF64 P;
    bool ready = false;  // warp-uniform
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        const int l1 = (pass ? b1 : a1) * M;
#pragma unroll 1
        for (int l = (pass ? b0 : a0) * M; l < l1; ++l) {
            const dbl4 ln = lines64[l];
            const double rs = rc.x * ln.x + rc.y * ln.y + rc.z * ln.z;
            const bool near_line = !(rc2 - rs * rs > bound);
            if (!__any_sync(0xffffffffu, near_line)) continue;
            if (!ready) {
                pair_setup_f64(P, x, r, vertex_index(x, r));
                ready = true;
            }
            if (near_line && line_f64(P, ln, acc)) ++hits;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kRayThreads, 4) ray_kernel(const VelocityArgs a)
{
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int RB = ray_rec_bytes<T>();
    constexpr int STAGE = kRayTile * RB;
    constexpr int NW = kRayThreads / 32;

    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *stages = smem;                                               // [S][TILE * RB]
    float *spts = reinterpret_cast<float *>(smem + kRayStages * STAGE);          // [threads][9] float splits
    RayPipe *pipe = reinterpret_cast<RayPipe *>(spts + 9 * kRayThreads);
    MeshDesc *s_md = reinterpret_cast<MeshDesc *>(reinterpret_cast<unsigned char *>(pipe) + 64);
    int64_t *s_item = reinterpret_cast<int64_t *>(reinterpret_cast<unsigned char *>(s_md) + 256);
    T *sz = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(s_item) + 16);  // [n_phi] cos(phi_n)
    float4 *sdir = reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(sz) + 16 * ((sizeof(T) * 256 + 15) / 16));

    if (a.skip && *a.skip) return;  // the mesh walk evaluated these points
    const int tid = threadIdx.x, lane = tid & 31;
    const int N = a.lines.n_phi, M = a.lines.n_theta;
    // cos(phi_n) of each ring (descending in n) and, for float32, the direction table
    for (int n = tid; n < N; n += kRayThreads) sz[n] = (T)a.lines.f64[n * M].z;
    // the float32 direction table in shared memory (the host sends larger tables to the velocity kernel)
    if (F32)
        for (int l = tid; l < a.L; l += kRayThreads) sdir[l] = a.lines.f32[l];
    if (tid == 0) {
        for (int st = 0; st < kRayStages; ++st) {
            mbar_init(&pipe->full[st], 1);
            pipe->done[st] = 0;
        }
        fence_mbar_init();
    }
    __syncthreads();
    const MeshDesc &md = *s_md;
    uint32_t phase = 0u;

    auto issue = [&](int64_t t, int st) {
        const int64_t first = t * kRayTile;
        const int cnt = (int)min((int64_t)kRayTile, md.n_tets - first);
        const uint32_t bytes = (uint32_t)cnt * RB;
        const void *src = F32 ? (const void *)(md.near32 + first * kNearF32Vec4)
                              : (const void *)(md.near64 + first * kNearF64);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&pipe->full[st], bytes);
        if (a.withhold_copies) return;
        bulk_g2s(stages + st * STAGE, src, bytes, &pipe->full[st]);
    };
    const long long wait_cap = a.wait_polls > 0 ? a.wait_polls : kWaitCap;

    for (;;) {
        if (tid == 0) {
            int64_t item = atomicAdd(a.work_counter, 1ull);
            if (item < a.n_items) {
                *s_md = a.m;
            } else {
                item = -1;
            }
            *s_item = item;
        }
        __syncthreads();
        const int64_t item = *s_item;
        if (item < 0) break;
        const int64_t k = md.k;
        const int64_t n_blocks = (k + kRayThreads - 1) / kRayThreads;
        const int64_t n_tiles = (md.n_tets + kRayTile - 1) / kRayTile;
        const int64_t pb = item % n_blocks, ck = item / n_blocks;
        const int64_t t0 = ck * md.tiles_per_chunk;
        const int64_t t1 = min(t0 + (int64_t)md.tiles_per_chunk, n_tiles);
        const int n_local = (int)(t1 - t0);

        if (tid == 0)
            for (int i = 0; i < kRayStages && i < n_local; ++i) issue(t0 + i, i);

        int64_t gi = pb * kRayThreads + tid;
        const bool valid = gi < k;
        if (!valid) gi = k - 1;  // pad with a real point; its result is not written
        const int64_t src = md.perm[gi];
        float *xs = spts + 9 * tid;
#pragma unroll
        for (int j = 0; j < 3; ++j) split3(md.pts[3 * src + j], xs[3 * j], xs[3 * j + 1], xs[3 * j + 2]);
        const V3<double> xd = mk(md.pts[3 * src], md.pts[3 * src + 1], md.pts[3 * src + 2]);
        // bounding ball of the warp's 32 points (float, padded): the direction windows are the warp's
        float cwx, cwy, cwz, rw;
        {
            float mnx = xs[0], mxx = mnx, mny = xs[3], mxy = mny, mnz = xs[6], mxz = mnz;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
                mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
                mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, o));
                mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
                mnz = fminf(mnz, __shfl_xor_sync(0xffffffffu, mnz, o));
                mxz = fmaxf(mxz, __shfl_xor_sync(0xffffffffu, mxz, o));
            }
            cwx = 0.5f * (mnx + mxx);
            cwy = 0.5f * (mny + mxy);
            cwz = 0.5f * (mnz + mxz);
            const float ex = mxx - mnx, ey = mxy - mny, ez = mxz - mnz;
            rw = 0.5f * sqrtf(ex * ex + ey * ey + ez * ez) * 1.001f + 1e-6f;
        }

        float ks[3] = {0.f, 0.f, 0.f}, kc[3] = {0.f, 0.f, 0.f};  // float32: Kahan sum across tiles
        V3<double> acc64 = mk(0.0, 0.0, 0.0);                    // float64: plain sum
        int hits = 0;
        bool aborted = false;
#pragma unroll 1
        for (int i = 0; i < n_local; ++i) {
            const int st = i % kRayStages;
            const int64_t t = t0 + i;
            // the warp gives up as one (a lane that saw the copy land leaves with the others)
            if (!__all_sync(0xffffffffu, mbar_wait(&pipe->full[st], (phase >> st) & 1u, wait_cap))) {
                aborted = true;
                break;
            }
            phase ^= 1u << st;
            const int cnt = (int)min((int64_t)kRayTile, md.n_tets - t * kRayTile);
            const unsigned char *tb = stages + st * STAGE;
            if constexpr (F32) {
                float ax = 0.f, ay = 0.f, az = 0.f;
                uint32_t redo_tets = 0u;  // this lane's tets of the tile that need float64 steps
#pragma unroll 1
                for (int j = 0; j < cnt; ++j) {
                    const float4 *r32 = reinterpret_cast<const float4 *>(tb) + j * kNearF32Vec4;
                    const float4 ch = r32[nf32::CH];
                    int a0, a1, b0, b1;
                    ring_window<float>(sz, N, mk(ch.x - cwx, ch.y - cwy, ch.z - cwz), rw,
                                       r32[nf32::G2].w * (1.0f + kBoundPadF), a0, a1, b0, b1);
                    if (ray_tet_f32(xs, r32, sdir, M, a0, a1, b0, b1, ax, ay, az, hits)) redo_tets |= 1u << j;
                }
                // the float64 steps of the tile (rare), while its records are still staged
#pragma unroll 1
                while (redo_tets) {
                    const int j = __ffs(redo_tets) - 1;
                    redo_tets &= redo_tets - 1u;
                    const float4 *r32 = reinterpret_cast<const float4 *>(tb) + j * kNearF32Vec4;
                    const float4 ch = r32[nf32::CH];
                    int a0, a1, b0, b1;
                    ring_window<float>(sz, N, mk(ch.x - cwx, ch.y - cwy, ch.z - cwz), rw,
                                       r32[nf32::G2].w * (1.0f + kBoundPadF), a0, a1, b0, b1);
                    ray_tet_redo_f64(xs, r32, md.near64 + (t * kRayTile + j) * kNearF64, sdir, a.lines.f64, M, a0,
                                     a1, b0, b1, ax, ay, az, hits);
                }
                const float v[3] = {ax, ay, az};
#pragma unroll
                for (int jj = 0; jj < 3; ++jj) {
                    const float y = v[jj] - kc[jj];
                    const float s2 = ks[jj] + y;
                    kc[jj] = (s2 - ks[jj]) - y;
                    ks[jj] = s2;
                }
            } else {
#pragma unroll 1
                for (int j = 0; j < cnt; ++j) {
                    const double *r = reinterpret_cast<const double *>(tb) + j * kNearF64;
                    int a0, a1, b0, b1;
                    ring_window<double>(sz, N, mk(r[nf64::C] - cwx, r[nf64::C + 1] - cwy, r[nf64::C + 2] - cwz),
                                        (double)rw, r[nf64::RB2] * (1.0 + kBoundPadD), a0, a1, b0, b1);
                    ray_tet_f64(xd, r, a.lines.f64, M, a0, a1, b0, b1, acc64, hits);
                }
            }
            // this warp is done with stage st; the last warp to finish refills it
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                const int prev = atomicAdd(&pipe->done[st], 1);
                if (prev == NW - 1) {
                    pipe->done[st] = 0;
                    __threadfence_block();
                    if (i + kRayStages < n_local) issue(t + kRayStages, st);
                }
            }
        }
        if (aborted) {
            if (tid == 0) atomicOr(a.flag, kFlagTimeout);
            mbar_drain<kRayStages>(pipe->full, phase, wait_cap);
            return;
        }
        if (valid) {
            double *dst = md.partial + (ck * k + gi) * 3;
            if constexpr (F32) {
#pragma unroll
                for (int jj = 0; jj < 3; ++jj) dst[jj] = (double)ks[jj] - (double)kc[jj];
            } else {
                dst[0] = acc64.x;
                dst[1] = acc64.y;
                dst[2] = acc64.z;
            }
            if (a.counts) {
                const int64_t ntets_chunk = min(md.n_tets, t1 * kRayTile) - t0 * kRayTile;
                atomicAdd(&a.counts[3 * src + 0], (int)ntets_chunk);
                atomicAdd(&a.counts[3 * src + 2], hits);
            }
        }
        __syncthreads();  // stages and points are reused by the next item
    }
}

__global__ void ray_zero_kernel(int32_t *counts, int64_t n, unsigned long long *work_counter, const int *skip)
{
    if (skip && *skip) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) *work_counter = 0ull;
    if (counts && i < n) counts[i] = 0;
}

template <typename T>
size_t ray_smem_bytes(int lines_in_smem)
{
    return (size_t)kRayStages * kRayTile * ray_rec_bytes<T>() + sizeof(float) * 9 * kRayThreads + 64 + 256 + 16 +
           16 * ((sizeof(T) * 256 + 15) / 16) + sizeof(float4) * (size_t)lines_in_smem;
}

template <typename T>
cudaError_t ray_launch_t(const VelocityArgs &a, int n_sm, cudaStream_t st, int *grid_out, int *occ_out, bool query)
{
    auto kern = ray_kernel<T>;
    const size_t sm = ray_smem_bytes<T>(sizeof(T) == 4 ? a.L : 0);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRayThreads, sm);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (occ_out) *occ_out = occ;
    if (query) return cudaSuccess;
    const int64_t grid = std::min<int64_t>(a.n_items, (int64_t)n_sm * occ);
    if (grid_out) *grid_out = (int)grid;
    kern<<<(unsigned)grid, kRayThreads, sm, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

LaunchShape ray_shape()
{
    LaunchShape s;
    s.threads = kRayThreads;
    s.points_per_thread = 1;
    s.tile = kRayTile;
    return s;
}

int ray_ctas_per_sm(int precision, int L)
{
    VelocityArgs q;
    q.L = L;
    q.smem_lines = 1;
    int occ = 0;
    if (precision == BS_FP32) ray_launch_t<float>(q, 1, 0, nullptr, &occ, true);
    else ray_launch_t<double>(q, 1, 0, nullptr, &occ, true);
    return occ;
}

cudaError_t launch_ray(int precision, const VelocityArgs &a, int n_sm, cudaStream_t st, int *grid_out,
                       cudaEvent_t ev_start, cudaEvent_t ev_stop)
{
    const int64_t nc = a.counts ? 3 * a.m.k : 0;
    ray_zero_kernel<<<(unsigned)((nc + 255) / 256 + 1), 256, 0, st>>>(a.counts, nc, a.work_counter, a.skip);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev_start && (e = cudaEventRecord(ev_start, st)) != cudaSuccess) return e;
    e = precision == BS_FP32 ? ray_launch_t<float>(a, n_sm, st, grid_out, nullptr, false)
                             : ray_launch_t<double>(a, n_sm, st, grid_out, nullptr, false);
    if (e != cudaSuccess) return e;
    if (ev_stop) e = cudaEventRecord(ev_stop, st);
    return e;
}

}  // namespace bs
