// bs_walk.cu -- the all-ray velocity at the mesh's own nodes by walking each line through
// face-neighbour tets (the ray tracing through the mesh that the paper's conclusion, §4,
// proposes), instead of testing every tet against every line.
//
// At a node x every line x + t s of the direction table (Eq. 3) is split into the half-lines
// t > 0 along s and along -s.  A half-line leaves x through the incident tet whose face
// planes through x it enters (all g_i . d >= 0 for the faces i through x), then crosses the
// mesh tet by tet: in the current tet the chord [lo, hi] of the line is the one of the ray
// rule (barycentric clipping lambda_i = a_i + b_i t), the line leaves through the face that
// attains hi, and the next tet is the face neighbour across it, until the line leaves the
// mesh.  Each visited tet contributes its chord on the half-line, so the sum over both
// half-lines is the ray rule's sum over all tets (Eq. 5 with sign(t)): with I(d) the integral
// of omega along the half-line in direction d, J = I(s) - I(-s).  On a convex domain every line
// leaves the mesh once.  After every change of the node positions the library checks that every
// boundary node lies on the inner side of every boundary face's plane; where that fails (a
// non-convex domain) a line that leaves the mesh is followed through a uniform grid of the
// boundary faces to the face where it comes back in, if any, and the walk goes on from there.
// The walk needs a conforming mesh whose nodes all belong to some tet; otherwise the all-ray
// kernel evaluates the nodes.  The paths are all queued and each returns at once when another
// one is in charge, so nothing waits on the host.
//
// Derivative along a direction e (the stretching term (omega . grad) v of the Lagrangian method with
// e = omega): per half-line dI/de = sum over the tets it crosses of the chord length on the
// half-line times e . grad omega_T, plus omega(exit) dT/de where the line leaves the mesh
// (omega jumps to zero there; T is the exit parameter, dT/de = -(g_f . e)/(g_f . d) for the
// boundary face f with barycentric gradient g_f); inside the mesh omega is continuous and the
// chord ends of neighbouring tets cancel.  dv/de = sum over lines k s x (dI(s) - dI(-s)).
//
// One warp per node, the lanes over the lines; per-node sums by warp reduction (no atomics,
// deterministic).  The float32 walk reads one 128-byte record per tet step (gradients, longest
// edge, vertex 0 as float splits, nodal vorticity, the four face neighbours: everything a step
// needs in one cache line), rebuilt from the near records after every mesh update.  A walk that has not left the mesh after max_steps tets (it cannot happen on
// a valid mesh) sets the error flag and stops.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <tuple>
#include <vector>

#include "bs_internal.cuh"
#include "bs_near.cuh"

namespace bs {
namespace {

constexpr int kWalkThreads = 128;     // 4 nodes per CTA
constexpr float kStartTolF = 1e-6f;   // a half-line whose best start margin is below -tol leaves the mesh at x
constexpr double kStartTolD = 1e-12;

// First boundary face through which the line x + t d enters the mesh at some t > t0 (the line is
// outside the mesh just after t0), or -1.  A 3-D DDA over the uniform grid of boundary faces from
// where the line enters the grid's box; in each cell, Moller-Trumbore against the cell's faces
// (a face is an entry when d points against its outward normal); the nearest entry within the
// cells visited so far ends the search once the line has left the cell holding it.  The search
// visits at most 3G + 3 cells.
// Clip of the line to the slab [lo, hi] of one axis (tin, tout narrowed); false when the line misses it.
template <typename T>
__device__ __forceinline__ bool slab(T x, T d, T lo, T hi, T &tin, T &tout)
{
    if (d == (T)0) return x >= lo && x <= hi;
    const T t1 = (lo - x) / d, t2 = (hi - x) / d;
    tin = max(tin, min(t1, t2));
    tout = min(tout, max(t1, t2));
    return true;
}

// DDA set-up along one axis: cell index, step, parameter of the next cell boundary and per-cell increment.
template <typename T>
__device__ __forceinline__ void dda_axis(T x, T d, T tin, T lo, T cell, T inv, int G, int &i, int &st, T &tmax,
                                        T &tdelta)
{
    i = min(G - 1, max(0, (int)floor((x + tin * d - lo) * inv)));
    if (d > (T)0) {
        st = 1;
        tmax = (lo + (i + 1) * cell - x) / d;
        tdelta = cell / d;
    } else if (d < (T)0) {
        st = -1;
        tmax = (lo + i * cell - x) / d;
        tdelta = -cell / d;
    } else {
        st = 0;
        tmax = (T)INFINITY;
        tdelta = (T)INFINITY;
    }
}

// T = float for the float32 walk (the float copy of the grid and the faces), double for the float64 walk.
template <typename T>
__device__ __forceinline__ int walk_reenter(const WalkArgs &a, V3<T> x, V3<T> d, T t0, T &t_hit)
{
    constexpr bool F = sizeof(T) == 4;
    const WalkGrid &g = *a.grid;
    const int G = g.G;
    const T lo0 = F ? (T)g.lo32[0] : (T)g.lo[0], lo1 = F ? (T)g.lo32[1] : (T)g.lo[1], lo2 = F ? (T)g.lo32[2] : (T)g.lo[2];
    const T c0 = F ? (T)g.cell32[0] : (T)g.cell[0], c1 = F ? (T)g.cell32[1] : (T)g.cell[1],
            c2 = F ? (T)g.cell32[2] : (T)g.cell[2];
    const T i0 = F ? (T)g.inv32[0] : (T)g.inv[0], i1 = F ? (T)g.inv32[1] : (T)g.inv[1], i2 = F ? (T)g.inv32[2] : (T)g.inv[2];
    T tin = t0, tout = (T)INFINITY;
    if (!slab<T>(x.x, d.x, lo0, lo0 + G * c0, tin, tout) || !slab<T>(x.y, d.y, lo1, lo1 + G * c1, tin, tout) ||
        !slab<T>(x.z, d.z, lo2, lo2 + G * c2, tin, tout) || !(tin <= tout))
        return -1;
    int ix, iy, iz, sx, sy, sz;
    T mx, my, mz, dx, dy, dz;
    dda_axis<T>(x.x, d.x, tin, lo0, c0, i0, G, ix, sx, mx, dx);
    dda_axis<T>(x.y, d.y, tin, lo1, c1, i1, G, iy, sy, my, dy);
    dda_axis<T>(x.z, d.z, tin, lo2, c2, i2, G, iz, sz, mz, dz);
    const T eps = F ? (T)1e-6 : (T)1e-14;  // relative: entries at or before t0 are not entries
    const T tmin = t0 + eps * max((T)1, fabs(t0));
    const T tol = F ? (T)1e-6 : (T)1e-12;  // area-coordinate tolerance
    T best = (T)INFINITY;
    int bf = -1;
    for (int it = 0; it < 3 * G + 3; ++it) {
        const int c = (iz * G + iy) * G + ix;
        for (int j = a.cell_off[c]; j < a.cell_off[c + 1]; ++j) {
            const int f = a.cell_face[j];
            V3<T> p0, e1, e2;
            if constexpr (F) {
                const float *q = a.bgeo32 + (int64_t)f * kBFaceGeo;
                p0 = mk(q[0], q[1], q[2]);
                e1 = mk(q[3], q[4], q[5]);
                e2 = mk(q[6], q[7], q[8]);
            } else {
                const double *q = a.bgeo + (int64_t)f * kBFaceGeo;
                p0 = mk(q[0], q[1], q[2]);
                e1 = mk(q[3], q[4], q[5]);
                e2 = mk(q[6], q[7], q[8]);
            }
            const V3<T> n = mk(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
            const T nd = dot3(n, d);
            if (!(nd < (T)0)) continue;  // not an entry (outward normal e1 x e2)
            // the plane's crossing first: a face behind tmin or beyond the best entry so far needs no more
            const T tp = (n.x * (p0.x - x.x) + n.y * (p0.y - x.y) + n.z * (p0.z - x.z)) / nd;
            if (!(tp > tmin - tol * max((T)1, fabs(tmin))) || !(tp < best + tol * max((T)1, fabs(tp)))) continue;
            const V3<T> P = mk(d.y * e2.z - d.z * e2.y, d.z * e2.x - d.x * e2.z, d.x * e2.y - d.y * e2.x);
            const T det = dot3(e1, P);
            if (fabs(det) <= (F ? (T)1e-7 : (T)1e-14) * sqrt(dot3(e1, e1) * dot3(e2, e2))) continue;
            const T inv = (T)1 / det;
            const V3<T> Tv = mk(x.x - p0.x, x.y - p0.y, x.z - p0.z);
            const T u = dot3(Tv, P) * inv;
            if (u < -tol || u > (T)1 + tol) continue;
            const V3<T> Qv = mk(Tv.y * e1.z - Tv.z * e1.y, Tv.z * e1.x - Tv.x * e1.z, Tv.x * e1.y - Tv.y * e1.x);
            const T v = dot3(d, Qv) * inv;
            if (v < -tol || u + v > (T)1 + tol) continue;
            const T t = dot3(e2, Qv) * inv;
            if (t > tmin && t < best) {
                best = t;
                bf = f;
            }
        }
        const T tnext = min(mx, min(my, mz));
        if (bf >= 0 && best <= tnext) break;  // nothing nearer can lie in a later cell
        if (tnext > tout) break;
        if (mx <= my && mx <= mz) {
            ix += sx;
            mx += dx;
            if (ix < 0 || ix >= G) break;
        } else if (my <= mz) {
            iy += sy;
            my += dy;
            if (iy < 0 || iy >= G) break;
        } else {
            iz += sz;
            mz += dz;
            if (iz < 0 || iz >= G) break;
        }
    }
    t_hit = best;
    return bf;
}

// Start tets of the two half-lines along +s and -s from a node: the incident tet whose face planes through x
// the half-line enters, by the largest margin min over those faces of (g_i . d) / |g_i| (first in incidence
// order on a tie).  One pass serves both directions (the margins along -s are the negated products), reading
// the incident tets' face gradients and their reciprocal norms from the warp's staged copy (count <=
// kWalkIncCap) or, for a node with more incident tets, from the walk records.
// two consecutive float4 of read-only global memory in one 256-bit load (p 32-byte aligned)
__device__ __forceinline__ void ldg_v8(const float4 *p, float4 &a, float4 &b)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

constexpr int kWalkIncCap = 64;  // incident tets staged in shared memory per node
// face j (0..2) of the three through vertex k (faces i != k, ascending): its gradient and reciprocal norm,
// from the walk record's g1..g3 (g0 = -(g1 + g2 + g3)); selects, no indexed register arrays
__device__ __forceinline__ float4 face_through(float4 q0, float4 q1, float4 q2, int k, int j)
{
    const int i = j + (j >= k ? 1 : 0);
    const V3<float> g = i == 0 ? mk(-(q0.x + q1.x + q2.x), -(q0.y + q1.y + q2.y), -(q0.z + q1.z + q2.z))
                        : i == 1 ? mk(q0.x, q0.y, q0.z)
                        : i == 2 ? mk(q1.x, q1.y, q1.z)
                                 : mk(q2.x, q2.y, q2.z);
    return make_float4(g.x, g.y, g.z, rsqrtf(dot3(g, g)));
}
struct WalkStart {
    int T = -1, k = -1;
    float best = -INFINITY;
};
__device__ __forceinline__ void walk_start_f32(const WalkArgs &a, int64_t node, const float4 *sg, const int *scode,
                                               int n_staged, V3<float> s, WalkStart &wp, WalkStart &wm)
{
    const int e0 = a.inc_off[node], n = a.inc_off[node + 1] - e0;
    for (int e = 0; e < n; ++e) {
        int code;
        float4 f[3];  // the three faces through x: gradient and reciprocal norm
        if (n_staged >= 0) {
            code = scode[e];
            f[0] = sg[3 * e];
            f[1] = sg[3 * e + 1];
            f[2] = sg[3 * e + 2];
        } else {
            code = a.inc[e0 + e];
            const float4 *r = a.wrec + (int64_t)(code >> 2) * kWalkRecVec4;
            const float4 q0 = __ldg(r), q1 = __ldg(r + 1), q2 = __ldg(r + 2);
#pragma unroll
            for (int j = 0; j < 3; ++j) f[j] = face_through(q0, q1, q2, code & 3, j);
        }
        float mp = INFINITY, mm = INFINITY;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float p = dot3(mk(f[j].x, f[j].y, f[j].z), s) * f[j].w;
            mp = fminf(mp, p);
            mm = fminf(mm, -p);
        }
        if (mp > wp.best) {
            wp.best = mp;
            wp.T = code >> 2;
            wp.k = code & 3;
        }
        if (mm > wm.best) {
            wm.best = mm;
            wm.T = code >> 2;
            wm.k = code & 3;
        }
    }
}

// The integral of omega along one half-line x + t d, t > 0, walking the tets from node `node`, starting in
// st.T (x is its vertex st.k).  float32: the point as float splits (xh, xm); records from near32.
template <bool GRAD, bool RE, bool NEAR>
__device__ V3<float> walk_f32(const WalkArgs &a, WalkStart st, V3<double> xd, const float xh[3],
                              const float xm[3], V3<float> d, V3<float> e, V3<float> &dI, int &hits, float r_stop)
{
    V3<float> I = mk(0.f, 0.f, 0.f);
    int T = st.T, kk = st.k;
    const float best = st.best;
    bool exact = true;  // x is vertex kk of T
    int entf = -1;      // face of T through which the line came in from outside the mesh
    float tcur = 0.f;  // the farthest point reached: re-entries are looked for beyond it only, so that a line
                       // grazing a fold, where the tet tests and the face search round differently, cannot cycle
    const V3<float> xf = mk((float)xd.x, (float)xd.y, (float)xd.z);
    int prevT = -1;  // the tet the line came from (-1 at the start and after coming back in from outside)
    if (T < 0 || best < -kStartTolF) {  // the half-line leaves the mesh at x
        if constexpr (!RE) return I;
        float th;  // a non-convex mesh: the line may come back
        const int f = walk_reenter<float>(a, xf, d, 0.f, th);
        if (f < 0) return I;
        T = a.bface[f] >> 2;
        entf = a.bface[f] & 3;
        exact = false;
        tcur = th;
    }
    for (int step = 0; T >= 0; ++step) {
        if (step >= a.max_steps) {
            atomicOr(a.flag, kFlagWalk);
            break;
        }
        const float4 *r = a.wrec + (int64_t)T * kWalkRecVec4;
        // the record in five loads, 32 bytes where the registers allow (a gather: one L1 wavefront per lane and
        // load, so the fewer loads the better); the vorticities further down
        float4 q0, q1, q2, q3;
        ldg_v8(r, q0, q1);
        ldg_v8(r + 2, q2, q3);
        const int4 nb = __ldg(reinterpret_cast<const int4 *>(r + 7));  // the face neighbours
        // the face the line came in through (from the previous tet, or from outside): never left through again
        const int inface = prevT >= 0 ? (nb.x == prevT ? 0 : nb.y == prevT ? 1 : nb.z == prevT ? 2 : 3) : entf;
        V3<float> g[4];
        g[1] = mk(q0.x, q0.y, q0.z);
        g[2] = mk(q1.x, q1.y, q1.z);
        g[3] = mk(q2.x, q2.y, q2.z);
        g[0] = mk(-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z));
        float av[4];
        if (exact) {
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = (i == kk) ? 1.0f : 0.0f;
        } else {
            // vertex 0 as float splits: hi = (q1.w, q2.w, q3.x), mid = (q3.y, q3.z, q3.w)
            const V3<float> d0 = mk((xh[0] - q1.w) + (xm[0] - q3.y), (xh[1] - q2.w) + (xm[1] - q3.z),
                                    (xh[2] - q3.x) + (xm[2] - q3.w));
            av[1] = dot3(g[1], d0);
            av[2] = dot3(g[2], d0);
            av[3] = dot3(g[3], d0);
            av[0] = 1.0f - av[1] - av[2] - av[3];
        }
        float b[4];
        b[1] = dot3(g[1], d);
        b[2] = dot3(g[2], d);
        b[3] = dot3(g[3], d);
        b[0] = -(b[1] + b[2] + b[3]);
        // chord [lo, hi] exactly as the ray rule takes it (its contribution); the way on: the nearest face ahead
        // other than the one the line came in through (hx, exitf), so that two tets that round a nearly
        // parallel shared face differently cannot hand the line back and forth
        float lo = -INFINITY, hi = INFINITY, hx = INFINITY;
        int exitf = -1;
        bool empty = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (b[i] * b[i] <= kParF * kParF * dot3(g[i], g[i])) {
                empty = empty || (av[i] < -kParF);
            } else {
                const float ti = -av[i] / b[i];
                if (b[i] > 0.f) {
                    lo = fmaxf(lo, ti);
                } else {
                    hi = fminf(hi, ti);
                    if (i != inface && ti < hx) {
                        hx = ti;
                        exitf = i;
                    }
                }
            }
        }
        if (exitf < 0) {  // no face ahead: not a bounded tet along this line
            atomicOr(a.flag, kFlagWalkStuck);
            break;
        }
        bool take = true;  // near mode: only the tets the far sweep left out (it takes the others)
        if constexpr (NEAR) {
            if (fmaxf(lo, 0.f) > r_stop) break;  // this tet and every one beyond are far from the node
            const float4 o = __ldg(a.tile_hdr + 2 * (T / a.tile));
            const float4 c = __ldg(reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(a.far) +
                                                                    (int64_t)T * a.far_stride));
            take = pair_is_near_f32(xh[0] - o.x, xh[1] - o.y, xh[2] - o.z, c, a.far_ratio2_f);
        }
        // omega at the vertices (w0 w1 w2 w3, 12 floats)
        float4 q4, q5;
        ldg_v8(r + 4, q4, q5);
        const float4 q6 = __ldg(r + 6);
        float ge[4];  // g_i . e
        if constexpr (GRAD) {
            ge[1] = dot3(g[1], e);
            ge[2] = dot3(g[2], e);
            ge[3] = dot3(g[3], e);
            ge[0] = -(ge[1] + ge[2] + ge[3]);
        }
        if (take && !empty && hi - lo > (float)kTau * q0.w) {
            const float l0 = fmaxf(lo, 0.f);
            const float f1 = hi - l0, f2 = 0.5f * (hi * hi - l0 * l0);
            const float c0 = f1 * av[0] + f2 * b[0], c1 = f1 * av[1] + f2 * b[1];
            const float c2 = f1 * av[2] + f2 * b[2], c3 = f1 * av[3] + f2 * b[3];
            I.x += c0 * q4.x + c1 * q4.w + c2 * q5.z + c3 * q6.y;
            I.y += c0 * q4.y + c1 * q5.x + c2 * q5.w + c3 * q6.z;
            I.z += c0 * q4.z + c1 * q5.y + c2 * q6.x + c3 * q6.w;
            if constexpr (GRAD) {  // chord length times e . grad omega_T
                dI.x += f1 * (ge[0] * q4.x + ge[1] * q4.w + ge[2] * q5.z + ge[3] * q6.y);
                dI.y += f1 * (ge[0] * q4.y + ge[1] * q5.x + ge[2] * q5.w + ge[3] * q6.z);
                dI.z += f1 * (ge[0] * q4.z + ge[1] * q5.y + ge[2] * q6.x + ge[3] * q6.w);
            }
            ++hits;
        }
        const int next = exitf == 0 ? nb.x : exitf == 1 ? nb.y : exitf == 2 ? nb.z : nb.w;
        if constexpr (GRAD) {
            // where omega jumps (the line enters from outside at lo, or leaves at hi): omega there times the
            // shift of that point, dT/de = -(g_f . e)/b_f; the face's g . e and b picked without indexing the
            // arrays (they stay in registers)
            for (int side = 0; side < 2; ++side) {
                const int f = side == 0 ? entf : (next < 0 ? exitf : -1);
                if (f < 0) continue;
                const float tt = side == 0 ? lo : hx;
                const float c0 = av[0] + b[0] * tt, c1 = av[1] + b[1] * tt;
                const float c2 = av[2] + b[2] * tt, c3 = av[3] + b[3] * tt;
                const float gef = f == 0 ? ge[0] : f == 1 ? ge[1] : f == 2 ? ge[2] : ge[3];
                const float bf = f == 0 ? b[0] : f == 1 ? b[1] : f == 2 ? b[2] : b[3];
                const float dT = (side == 0 ? gef : -gef) / bf;  // entry: -omega dT/de; exit: +omega dT/de
                dI.x += dT * (c0 * q4.x + c1 * q4.w + c2 * q5.z + c3 * q6.y);
                dI.y += dT * (c0 * q4.y + c1 * q5.x + c2 * q5.w + c3 * q6.z);
                dI.z += dT * (c0 * q4.z + c1 * q5.y + c2 * q6.x + c3 * q6.w);
            }
        }
        exact = false;
        entf = -1;
        prevT = T;
        if constexpr (RE) {
            tcur = fmaxf(tcur, hx);
            if (next == -2 && !(NEAR && tcur > r_stop)) {  // left through a face some boundary node lies beyond: does the line come back?
                float th;
                const int f = walk_reenter<float>(a, xf, d, tcur, th);
                if (f >= 0) {  // a grazing entry may give the tet an empty chord: never find it twice
                    T = a.bface[f] >> 2;
                    entf = a.bface[f] & 3;
                    prevT = -1;
                    tcur = fmaxf(tcur, th);
                    continue;
                }
            }
        }
        T = next;
    }
    return I;
}

// float64 form: records from near64.  Start tets as walk_start_f32, from float64 face gradients (staged as
// gradient and reciprocal norm, face j of the three through the node's vertex in ascending face order).
struct WalkStart64 {
    int T = -1, k = -1;
    double best = -INFINITY;
};
__device__ __forceinline__ void face_through64(const double *r, int k, int j, double out[4])
{
    const int i = j + (j >= k ? 1 : 0);
    V3<double> g;
    if (i == 0)
        g = mk(-(r[nf64::G] + r[nf64::G + 3] + r[nf64::G + 6]), -(r[nf64::G + 1] + r[nf64::G + 4] + r[nf64::G + 7]),
               -(r[nf64::G + 2] + r[nf64::G + 5] + r[nf64::G + 8]));
    else
        g = mk(r[nf64::G + 3 * i - 3], r[nf64::G + 3 * i - 2], r[nf64::G + 3 * i - 1]);
    out[0] = g.x;
    out[1] = g.y;
    out[2] = g.z;
    out[3] = 1.0 / sqrt(dot3(g, g));
}
__device__ __forceinline__ void walk_start_f64(const WalkArgs &a, int64_t node, const double *sg, const int *scode,
                                               int n_staged, V3<double> s, WalkStart64 &wp, WalkStart64 &wm)
{
    const int e0 = a.inc_off[node], n = a.inc_off[node + 1] - e0;
    for (int e = 0; e < n; ++e) {
        int code;
        double f[3][4];
        if (n_staged >= 0) {
            code = scode[e];
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) f[j][q] = sg[12 * e + 4 * j + q];
        } else {
            code = a.inc[e0 + e];
            const double *r = a.near64 + (int64_t)(code >> 2) * kNearF64;
#pragma unroll
            for (int j = 0; j < 3; ++j) face_through64(r, code & 3, j, f[j]);
        }
        double mp = INFINITY, mm = INFINITY;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double p = dot3(mk(f[j][0], f[j][1], f[j][2]), s) * f[j][3];
            mp = fmin(mp, p);
            mm = fmin(mm, -p);
        }
        if (mp > wp.best) {
            wp.best = mp;
            wp.T = code >> 2;
            wp.k = code & 3;
        }
        if (mm > wm.best) {
            wm.best = mm;
            wm.T = code >> 2;
            wm.k = code & 3;
        }
    }
}

template <bool GRAD, bool RE, bool NEAR>
__device__ V3<double> walk_f64(const WalkArgs &a, WalkStart64 st, V3<double> x, V3<double> d, V3<double> e,
                               V3<double> &dI, int &hits, double r_stop)
{
    V3<double> I = mk(0.0, 0.0, 0.0);
    int T = st.T, kk = st.k;
    const double best = st.best;
    bool exact = true;  // x is vertex kk of T
    int entf = -1;      // face of T through which the line came in from outside the mesh
    double tcur = 0.0;  // the farthest point reached (re-entries only beyond it)
    int prevT = -1;     // the tet the line came from
    if (T < 0 || best < -kStartTolD) {
        if constexpr (!RE) return I;
        double th;
        const int f = walk_reenter<double>(a, x, d, 0.0, th);
        if (f < 0) return I;
        T = a.bface[f] >> 2;
        entf = a.bface[f] & 3;
        exact = false;
        tcur = th;
    }
    for (int step = 0; T >= 0; ++step) {
        if (step >= a.max_steps) {
            atomicOr(a.flag, kFlagWalk);
            break;
        }
        const double *r = a.near64 + (int64_t)T * kNearF64;
        const int32_t *nbT = a.nbr + 4 * (int64_t)T;
        const int inface = prevT >= 0 ? (nbT[0] == prevT ? 0 : nbT[1] == prevT ? 1 : nbT[2] == prevT ? 2 : 3) : entf;
        V3<double> g[4];
        for (int i = 1; i < 4; ++i) g[i] = mk(r[nf64::G + 3 * i - 3], r[nf64::G + 3 * i - 2], r[nf64::G + 3 * i - 1]);
        g[0] = mk(-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z));
        double av[4];
        if (exact) {
            for (int i = 0; i < 4; ++i) av[i] = (i == kk) ? 1.0 : 0.0;
        } else {
            const V3<double> d0 = mk(x.x - r[nf64::V], x.y - r[nf64::V + 1], x.z - r[nf64::V + 2]);
            av[1] = dot3(g[1], d0);
            av[2] = dot3(g[2], d0);
            av[3] = dot3(g[3], d0);
            av[0] = 1.0 - av[1] - av[2] - av[3];
        }
        double b[4];
        b[1] = dot3(g[1], d);
        b[2] = dot3(g[2], d);
        b[3] = dot3(g[3], d);
        b[0] = -(b[1] + b[2] + b[3]);
        double lo = -INFINITY, hi = INFINITY, hx = INFINITY;  // chord as the rule takes it; the way on (hx, exitf)
        int exitf = -1;
        bool empty = false;
        for (int i = 0; i < 4; ++i) {
            if (b[i] * b[i] <= kParD * kParD * dot3(g[i], g[i])) {
                empty = empty || (av[i] < -kParD);
            } else {
                const double ti = -av[i] / b[i];
                if (b[i] > 0.0) {
                    lo = fmax(lo, ti);
                } else {
                    hi = fmin(hi, ti);
                    if (i != inface && ti < hx) {
                        hx = ti;
                        exitf = i;
                    }
                }
            }
        }
        if (exitf < 0) {
            atomicOr(a.flag, kFlagWalkStuck);
            break;
        }
        bool take = true;  // near mode: only the tets the far sweep left out
        if constexpr (NEAR) {
            if (fmax(lo, 0.0) > r_stop) break;
            take = pair_is_near_f64(x.x, x.y, x.z,
                                    reinterpret_cast<const double *>(a.far) + (int64_t)T * a.far_stride,
                                    a.far_ratio2);
        }
        double ge[4];  // g_i . e
        if constexpr (GRAD) {
            ge[1] = dot3(g[1], e);
            ge[2] = dot3(g[2], e);
            ge[3] = dot3(g[3], e);
            ge[0] = -(ge[1] + ge[2] + ge[3]);
        }
        if (take && !empty && hi - lo > kTau * r[nf64::H]) {
            const double l0 = fmax(lo, 0.0);
            const double f1 = hi - l0, f2 = 0.5 * (hi * hi - l0 * l0);
            for (int i = 0; i < 4; ++i) {
                const double c = f1 * av[i] + f2 * b[i];
                I.x += c * r[nf64::W + 3 * i];
                I.y += c * r[nf64::W + 3 * i + 1];
                I.z += c * r[nf64::W + 3 * i + 2];
                if constexpr (GRAD) {
                    dI.x += f1 * ge[i] * r[nf64::W + 3 * i];
                    dI.y += f1 * ge[i] * r[nf64::W + 3 * i + 1];
                    dI.z += f1 * ge[i] * r[nf64::W + 3 * i + 2];
                }
            }
            ++hits;
        }
        const int next = a.nbr[4 * (int64_t)T + exitf];
        if constexpr (GRAD) {
            for (int side = 0; side < 2; ++side) {  // omega jumps where the line enters or leaves the mesh
                const int f = side == 0 ? entf : (next < 0 ? exitf : -1);
                if (f < 0) continue;
                const double tt = side == 0 ? lo : hx;
                const double gef = f == 0 ? ge[0] : f == 1 ? ge[1] : f == 2 ? ge[2] : ge[3];
                const double bf = f == 0 ? b[0] : f == 1 ? b[1] : f == 2 ? b[2] : b[3];
                const double dT = (side == 0 ? gef : -gef) / bf;
                for (int i = 0; i < 4; ++i) {
                    const double c = dT * (av[i] + b[i] * tt);
                    dI.x += c * r[nf64::W + 3 * i];
                    dI.y += c * r[nf64::W + 3 * i + 1];
                    dI.z += c * r[nf64::W + 3 * i + 2];
                }
            }
        }
        exact = false;
        entf = -1;
        prevT = T;
        if constexpr (RE) {
            tcur = fmax(tcur, hx);
            if (next < 0 && !(NEAR && tcur > r_stop)) {
                double th;
                const int f = walk_reenter<double>(a, x, d, tcur, th);
                if (f >= 0) {
                    T = a.bface[f] >> 2;
                    entf = a.bface[f] & 3;
                    prevT = -1;
                    tcur = fmax(tcur, th);
                    continue;
                }
            }
        }
        T = next;
    }
    return I;
}

// RE: the instance for a non-convex domain (mode 2), with the re-entry search; the other one serves convex
// domains (mode 1).  Both are queued; the one not in charge returns at once.
// NEAR: the near field of the hybrid rule (see WalkArgs::near_mode), else the all-ray rule.
// The float32 instances for convex domains without the derivative are held to 64 registers (8 CTAs, 32 warps per
// SM): the walk waits on its dependent gathers, and the extra warps hide more of that than the few spills cost
// (256-mesh batch 223 -> 219 ms, all-ray 64^3 173 -> 164 ms).
template <typename T, bool GRAD, bool RE, bool NEAR>
__global__ void __launch_bounds__(kWalkThreads, (sizeof(T) == 4 && !GRAD && !RE) ? 8 : 1) walk_kernel(const WalkArgs a)
{
    const int mode = *a.mode;
    if (!mode) {  // not a conforming mesh: the all-ray kernel (or the near pass) takes the nodes
        if (GRAD && !RE && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.flag, kFlagNoWalk);  // no derivative
        return;
    }
    if ((mode == 2) != RE) return;
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * (kWalkThreads / 32) + (threadIdx.x >> 5);
    if (w >= a.n_nodes) return;  // whole warps
    const int64_t node = NEAR ? (int64_t)a.perm[w] : w;
    const T r_stop = NEAR ? (T)*a.r_stop : (T)0;
    const V3<double> xd = mk(a.nodes[3 * node], a.nodes[3 * node + 1], a.nodes[3 * node + 2]);
    const double *ep = a.dirs ? a.dirs + 3 * node : a.omega + 3 * node;
    const V3<double> ed = GRAD ? mk(ep[0], ep[1], ep[2]) : mk(0.0, 0.0, 0.0);
    T ax = 0, ay = 0, az = 0, gx = 0, gy = 0, gz = 0;
    int hits = 0;
    if constexpr (sizeof(T) == 4) {
        float xh[3], xm[3], xl;
        split3(xd.x, xh[0], xm[0], xl);
        split3(xd.y, xh[1], xm[1], xl);
        split3(xd.z, xh[2], xm[2], xl);
        const V3<float> e = mk((float)ed.x, (float)ed.y, (float)ed.z);
        // the node's incident tets, staged once for every line's start search: the gradients of the three faces
        // through x with their reciprocal norms, and the (tet, vertex) code
        __shared__ float4 s_inc[kWalkThreads / 32][3 * kWalkIncCap];
        __shared__ int s_code[kWalkThreads / 32][kWalkIncCap];
        const int wq = threadIdx.x >> 5;
        const int e0 = a.inc_off[node], n_inc = a.inc_off[node + 1] - e0;
        const int n_staged = n_inc <= kWalkIncCap ? n_inc : -1;  // warp-uniform
        for (int i = lane; i < n_staged; i += 32) {
            const int code = a.inc[e0 + i];
            const float4 *r = a.wrec + (int64_t)(code >> 2) * kWalkRecVec4;
            const float4 q0 = __ldg(r), q1 = __ldg(r + 1), q2 = __ldg(r + 2);
#pragma unroll
            for (int j = 0; j < 3; ++j) s_inc[wq][3 * i + j] = face_through(q0, q1, q2, code & 3, j);
            s_code[wq][i] = code;
        }
        __syncwarp();
        for (int l = lane; l < a.L; l += 32) {
            const float4 ln = __ldg(a.lines32 + l);
            const V3<float> s = mk(ln.x, ln.y, ln.z);
            V3<float> dp = mk(0.f, 0.f, 0.f), dm = mk(0.f, 0.f, 0.f);
            WalkStart sp, sm;
            walk_start_f32(a, node, s_inc[wq], s_code[wq], n_staged, s, sp, sm);
            const V3<float> Ip = walk_f32<GRAD, RE, NEAR>(a, sp, xd, xh, xm, s, e, dp, hits, r_stop);
            const V3<float> Im = walk_f32<GRAD, RE, NEAR>(a, sm, xd, xh, xm, mk(-s.x, -s.y, -s.z), e, dm, hits,
                                                          r_stop);
            const V3<float> J = mk(Ip.x - Im.x, Ip.y - Im.y, Ip.z - Im.z);
            ax += ln.w * (s.y * J.z - s.z * J.y);
            ay += ln.w * (s.z * J.x - s.x * J.z);
            az += ln.w * (s.x * J.y - s.y * J.x);
            if constexpr (GRAD) {
                const V3<float> D = mk(dp.x - dm.x, dp.y - dm.y, dp.z - dm.z);
                gx += ln.w * (s.y * D.z - s.z * D.y);
                gy += ln.w * (s.z * D.x - s.x * D.z);
                gz += ln.w * (s.x * D.y - s.y * D.x);
            }
        }
    } else {
        __shared__ double s_inc64[kWalkThreads / 32][12 * kWalkIncCap];
        __shared__ int s_code64[kWalkThreads / 32][kWalkIncCap];
        const int wq = threadIdx.x >> 5;
        const int e0 = a.inc_off[node], n_inc = a.inc_off[node + 1] - e0;
        const int n_staged = n_inc <= kWalkIncCap ? n_inc : -1;  // warp-uniform
        for (int i = lane; i < n_staged; i += 32) {
            const int code = a.inc[e0 + i];
            const double *r = a.near64 + (int64_t)(code >> 2) * kNearF64;
#pragma unroll
            for (int j = 0; j < 3; ++j) face_through64(r, code & 3, j, &s_inc64[wq][12 * i + 4 * j]);
            s_code64[wq][i] = code;
        }
        __syncwarp();
        for (int l = lane; l < a.L; l += 32) {
            const dbl4 ln = a.lines64[l];
            const V3<double> s = mk(ln.x, ln.y, ln.z);
            V3<double> dp = mk(0.0, 0.0, 0.0), dm = mk(0.0, 0.0, 0.0);
            WalkStart64 sp, sm;
            walk_start_f64(a, node, s_inc64[wq], s_code64[wq], n_staged, s, sp, sm);
            const V3<double> Ip = walk_f64<GRAD, RE, NEAR>(a, sp, xd, s, ed, dp, hits, r_stop);
            const V3<double> Im = walk_f64<GRAD, RE, NEAR>(a, sm, xd, mk(-s.x, -s.y, -s.z), ed, dm, hits, r_stop);
            const V3<double> J = mk(Ip.x - Im.x, Ip.y - Im.y, Ip.z - Im.z);
            ax += ln.w * (s.y * J.z - s.z * J.y);
            ay += ln.w * (s.z * J.x - s.x * J.z);
            az += ln.w * (s.x * J.y - s.y * J.x);
            if constexpr (GRAD) {
                const V3<double> D = mk(dp.x - dm.x, dp.y - dm.y, dp.z - dm.z);
                gx += ln.w * (s.y * D.z - s.z * D.y);
                gy += ln.w * (s.z * D.x - s.x * D.z);
                gz += ln.w * (s.x * D.y - s.y * D.x);
            }
        }
    }
    ax = warp_sum(ax);
    ay = warp_sum(ay);
    az = warp_sum(az);
    hits = warp_sum(hits);
    if constexpr (GRAD) {
        gx = warp_sum(gx);
        gy = warp_sum(gy);
        gz = warp_sum(gz);
    }
    if (NEAR && lane == 0) {  // the near totals by spatial position; the far sweep wrote the other counts
        a.near_out[3 * w] = (double)ax;
        a.near_out[3 * w + 1] = (double)ay;
        a.near_out[3 * w + 2] = (double)az;
        if (a.counts) a.counts[3 * node + 2] = hits;
    } else if (lane == 0) {
        a.out[3 * node] = (double)ax;
        a.out[3 * node + 1] = (double)ay;
        a.out[3 * node + 2] = (double)az;
        if constexpr (GRAD) {
            a.dout[3 * node] = (double)gx;
            a.dout[3 * node + 1] = (double)gy;
            a.dout[3 * node + 2] = (double)gz;
        }
        if (a.counts) {
            a.counts[3 * node] = (int32_t)min(a.n_tets, (int64_t)INT32_MAX);
            a.counts[3 * node + 1] = 0;
            a.counts[3 * node + 2] = hits;
        }
    }
}

__global__ void set_int_kernel(int *p, int v) { *p = v; }

// Box of the boundary nodes (one block), padded by 1e-6 of its largest extent, and a G^3 grid over it.
__global__ void grid_box_kernel(const double *__restrict__ nodes, const int32_t *__restrict__ bnode, int64_t n_bnode,
                                int G, WalkGrid *g)
{
    __shared__ double smn[3][256], smx[3][256];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = threadIdx.x; i < n_bnode; i += blockDim.x) {
        const int64_t q = bnode[i];
        for (int k = 0; k < 3; ++k) {
            mn[k] = fmin(mn[k], nodes[3 * q + k]);
            mx[k] = fmax(mx[k], nodes[3 * q + k]);
        }
    }
    for (int k = 0; k < 3; ++k) {
        smn[k][threadIdx.x] = mn[k];
        smx[k][threadIdx.x] = mx[k];
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; ++k) {
                smn[k][threadIdx.x] = fmin(smn[k][threadIdx.x], smn[k][threadIdx.x + o]);
                smx[k][threadIdx.x] = fmax(smx[k][threadIdx.x], smx[k][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double ext = 0.0;
        for (int k = 0; k < 3; ++k) ext = fmax(ext, smx[k][0] - smn[k][0]);
        const double pad = 1e-6 * ext + 1e-300;
        for (int k = 0; k < 3; ++k) {
            g->lo[k] = smn[k][0] - pad;
            g->cell[k] = (smx[k][0] - smn[k][0] + 2.0 * pad) / G;
            g->inv[k] = 1.0 / g->cell[k];
            g->lo32[k] = (float)g->lo[k];
            g->cell32[k] = (float)g->cell[k];
            g->inv32[k] = 1.0f / g->cell32[k];
        }
        g->G = G;
        g->ok = 1;
    }
}

// Per boundary face: its cells (those its bounding box overlaps).  Pass 0 counts the faces per cell and writes
// the face's record (vertex p0 and edges e1, e2 ordered so that e1 x e2 points out of the mesh); pass 1 fills
// the cells' face lists from the offsets (cell_cnt zeroed again in between).
template <int PASS>
__global__ void grid_faces_kernel(const double *__restrict__ nodes, const int32_t *__restrict__ tets,
                                  const int32_t *__restrict__ bface, int64_t n_bface, const WalkGrid *g,
                                  int32_t *cell_cnt, const int32_t *__restrict__ cell_off, int32_t *cell_face,
                                  int64_t cap, double *geo, float *geo32)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= n_bface) return;
    const int slot = bface[f];
    const int64_t t = slot >> 2;
    const int opp = slot & 3;
    int id[3], j = 0;
    for (int i = 0; i < 4; ++i)
        if (i != opp) id[j++] = tets[4 * t + i];
    V3<double> p[3];
    for (int i = 0; i < 3; ++i) p[i] = mk(nodes[3 * id[i]], nodes[3 * id[i] + 1], nodes[3 * id[i] + 2]);
    if (PASS == 0) {
        const int io = tets[4 * t + opp];
        const V3<double> po = mk(nodes[3 * io], nodes[3 * io + 1], nodes[3 * io + 2]);
        V3<double> e1 = mk(p[1].x - p[0].x, p[1].y - p[0].y, p[1].z - p[0].z);
        V3<double> e2 = mk(p[2].x - p[0].x, p[2].y - p[0].y, p[2].z - p[0].z);
        const V3<double> n = mk(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
        if (n.x * (po.x - p[0].x) + n.y * (po.y - p[0].y) + n.z * (po.z - p[0].z) > 0.0) {
            const V3<double> tmp = e1;
            e1 = e2;
            e2 = tmp;
        }
        double *q = geo + f * kBFaceGeo;
        q[0] = p[0].x; q[1] = p[0].y; q[2] = p[0].z;
        q[3] = e1.x; q[4] = e1.y; q[5] = e1.z;
        q[6] = e2.x; q[7] = e2.y; q[8] = e2.z;
        for (int i = 0; i < kBFaceGeo; ++i) geo32[f * kBFaceGeo + i] = (float)q[i];
    }
    const int G = g->G;
    int i0[3], i1[3];
    const double c[3][3] = {{p[0].x, p[1].x, p[2].x}, {p[0].y, p[1].y, p[2].y}, {p[0].z, p[1].z, p[2].z}};
    for (int k = 0; k < 3; ++k) {
        const double a = fmin(c[k][0], fmin(c[k][1], c[k][2])), b = fmax(c[k][0], fmax(c[k][1], c[k][2]));
        i0[k] = min(G - 1, max(0, (int)floor((a - g->lo[k]) * g->inv[k])));
        i1[k] = min(G - 1, max(0, (int)floor((b - g->lo[k]) * g->inv[k])));
    }
    for (int z = i0[2]; z <= i1[2]; ++z)
        for (int y = i0[1]; y <= i1[1]; ++y)
            for (int x = i0[0]; x <= i1[0]; ++x) {
                const int cell = (z * G + y) * G + x;
                if (PASS == 0) {
                    atomicAdd(&cell_cnt[cell], 1);
                } else {
                    const int64_t pos = (int64_t)cell_off[cell] + atomicAdd(&cell_cnt[cell], 1);
                    if (pos < cap) cell_face[pos] = (int32_t)f;
                }
            }
}

// Exclusive scan of the G^3 cell counts into cell_off (one block: a serial scan of each thread's run, then
// of the runs); the grid is not usable when the lists need more than cap entries.
__global__ void grid_scan_kernel(const int32_t *__restrict__ cnt, int n, int32_t *off, int64_t cap, WalkGrid *g)
{
    __shared__ int64_t run[1024];
    const int T = blockDim.x, tid = threadIdx.x;
    const int per = (n + T - 1) / T, b = tid * per, e = min(n, b + per);
    int64_t sum = 0;
    for (int i = b; i < e; ++i) sum += cnt[i];
    run[tid] = sum;
    __syncthreads();
    if (tid == 0) {
        int64_t acc = 0;
        for (int i = 0; i < T; ++i) {
            const int64_t v = run[i];
            run[i] = acc;
            acc += v;
        }
        off[n] = (int32_t)min(acc, (int64_t)INT32_MAX);
        if (acc > cap) g->ok = 0;
    }
    __syncthreads();
    int64_t acc = run[tid];
    for (int i = b; i < e; ++i) {
        off[i] = (int32_t)min(acc, (int64_t)INT32_MAX);
        acc += cnt[i];
    }
}

// A non-convex mesh (mode 2) whose face grid overflowed is left to the all-ray kernel (mode 0).
__global__ void grid_finalize_kernel(const WalkGrid *g, int *mode)
{
    if (*mode == 2 && !g->ok) *mode = 0;
}

// float32 walk record of a tet, one 128-byte line:
//   [g1 h] [g2 v0hi.x] [g3 v0hi.y] [v0hi.z v0mid.xyz] [w0.xyz w1.x] [w1.yz w2.xy] [w2.z w3.xyz] [nbr0..3]
__global__ void walk_records_kernel(const float4 *__restrict__ near32, const int32_t *__restrict__ nbr,
                                    int64_t n_tets, float4 *__restrict__ wrec)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_tets) return;
    const float4 *r = near32 + t * kNearF32Vec4;
    const float4 g1 = r[nf32::G1], g2 = r[nf32::G2], g3 = r[nf32::G3];
    const float4 w0 = r[nf32::W], w1 = r[nf32::W + 1], w2 = r[nf32::W + 2], w3 = r[nf32::W + 3];
    const float4 vh = r[nf32::VH], vm = r[nf32::VM];  // vertex 0 in .xyz
    float4 *o = wrec + t * kWalkRecVec4;
    o[0] = make_float4(g1.x, g1.y, g1.z, g1.w);
    o[1] = make_float4(g2.x, g2.y, g2.z, vh.x);
    o[2] = make_float4(g3.x, g3.y, g3.z, vh.y);
    o[3] = make_float4(vh.z, vm.x, vm.y, vm.z);
    o[4] = make_float4(w0.x, w0.y, w0.z, w1.x);
    o[5] = make_float4(w1.y, w1.z, w2.x, w2.y);
    o[6] = make_float4(w2.z, w3.x, w3.y, w3.z);
    o[7] = make_float4(__int_as_float(nbr[4 * t]), __int_as_float(nbr[4 * t + 1]), __int_as_float(nbr[4 * t + 2]),
                       __int_as_float(nbr[4 * t + 3]));
}

// mode = 1 iff every boundary node lies on the inner side of every boundary face's plane
// (within 1e-9 of the face's longest edge); mode must be set to the mesh's conformity (1 or 0)
// before the launch; a violation clears it.
// Every boundary face is checked (not only until the first violation): a face with a boundary node outside
// its plane is marked in the float32 walk record (neighbour -2 instead of -1), since a line can re-enter the
// mesh only after leaving it through such a face; a line that leaves through a face whose plane has the whole
// mesh on its inner side never comes back.
// A mesh of positive tets is folded when two tets that share a face lie on the same side of it (the
// tets overlap).  A line then need not leave a tet through the face it would in a valid mesh, and the
// walk is switched off (mode 0: the ray kernel serves the nodes).  One thread per interior face slot.
__global__ void fold_kernel(const double *__restrict__ nodes, const int32_t *__restrict__ tets,
                            const int32_t *__restrict__ nbr, int64_t n_tets, int *mode)
{
    const int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (slot >= 4 * n_tets) return;
    const int64_t t = slot >> 2, u = nbr[slot];
    if (u <= t) return;  // boundary face, or the pair is checked from the other side
    const int opp = (int)(slot & 3);
    int id[3], j = 0;
    for (int i = 0; i < 4; ++i)
        if (i != opp) id[j++] = tets[4 * t + i];
    int ou = -1;
    for (int i = 0; i < 4; ++i) {
        const int v = tets[4 * u + i];
        if (v != id[0] && v != id[1] && v != id[2]) ou = v;
    }
    if (ou < 0) return;
    const int ot = tets[4 * t + opp];
    const double *p0 = nodes + 3 * id[0], *p1 = nodes + 3 * id[1], *p2 = nodes + 3 * id[2];
    const double e1x = p1[0] - p0[0], e1y = p1[1] - p0[1], e1z = p1[2] - p0[2];
    const double e2x = p2[0] - p0[0], e2y = p2[1] - p0[1], e2z = p2[2] - p0[2];
    const double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    const double st = nx * (nodes[3 * ot] - p0[0]) + ny * (nodes[3 * ot + 1] - p0[1]) + nz * (nodes[3 * ot + 2] - p0[2]);
    const double su = nx * (nodes[3 * ou] - p0[0]) + ny * (nodes[3 * ou + 1] - p0[1]) + nz * (nodes[3 * ou + 2] - p0[2]);
    if ((st > 0.0 && su > 0.0) || (st < 0.0 && su < 0.0)) *mode = 0;
}

// Boundary nodes split into float pairs for the convexity screen: hi = (float)q, lo = (float)(q - hi) per
// coordinate, so that q = hi + lo to within 2^-48 |q|.  bpos[2 n_bnode].x receives (as bits) a float bound on
// every |coordinate| of the boundary nodes (positive floats order as their bit patterns).
__global__ void bnode_split_kernel(const double *__restrict__ nodes, const int32_t *__restrict__ bnode, int64_t n_bnode,
                                   float4 *__restrict__ bpos)
{
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_bnode; i += (int64_t)gridDim.x * blockDim.x) {
        const int q = bnode[i];
        float hi[3], lo[3];
        for (int k = 0; k < 3; ++k) {
            const double x = nodes[3 * q + k];
            hi[k] = (float)x;
            lo[k] = (float)(x - (double)hi[k]);
            m = fmaxf(m, __double2float_ru(fabs(x)));
        }
        bpos[2 * i] = make_float4(hi[0], hi[1], hi[2], 0.f);
        bpos[2 * i + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned *>(bpos + 2 * n_bnode), __float_as_uint(m));
}

constexpr int kConvexFaces = 128;  // faces per block (one per thread)
constexpr int kConvexTile = 256;   // boundary nodes per shared-memory tile

// Is every boundary node on the inner side of every boundary face's plane (within 1e-9 of the face's size)?
// Each thread holds one face; the block's nodes (a chunk of the boundary nodes, blockIdx.y) pass through shared
// memory in tiles.  The test n . (q - p0) <= tol is screened in float from the split coordinates: with
// d = (q_hi - p_hi) + (q_lo - p_lo) the screen's error is below 1e-6 sum |n_k d_k| + 2e-13 |n|_1 max|coord|
// (a few units of 2^-24 relative to the node's offset from the plane, plus the split's 2^-48 |q|), so a node
// whose screened value clears the threshold by that margin is inside; the rest are decided in float64.  A node
// that lies on the face's plane (equal coordinates along an axis-aligned face) gives d = 0 exactly and is
// decided by the screen.
__global__ void __launch_bounds__(kConvexFaces) convex_kernel(const double *__restrict__ nodes,
                                                             const int32_t *__restrict__ tets,
                                                             const int32_t *__restrict__ bface, int64_t n_bface,
                                                             const int32_t *__restrict__ bnode, int64_t n_bnode,
                                                             const float4 *__restrict__ bpos, int *mode, float4 *wrec)
{
    __shared__ float4 sh[2 * kConvexTile];
    if (*mode == 0) return;  // block-uniform: not conforming, or folded
    const int64_t f = blockIdx.x * (int64_t)kConvexFaces + threadIdx.x;
    const bool active = f < n_bface;
    V3<double> n = mk(0.0, 0.0, 0.0), p0 = mk(0.0, 0.0, 0.0);
    double tol = 0.0;
    int64_t t = 0;
    int opp = 0;
    float nxf = 0.f, nyf = 0.f, nzf = 0.f, tolf = 0.f, K = 0.f;
    float ph[3] = {0.f, 0.f, 0.f}, pl[3] = {0.f, 0.f, 0.f};
    if (active) {
        const int slot = bface[f];
        t = slot >> 2;
        opp = slot & 3;
        int id[3], j = 0;
        for (int i = 0; i < 4; ++i)
            if (i != opp) id[j++] = tets[4 * t + i];
        p0 = mk(nodes[3 * id[0]], nodes[3 * id[0] + 1], nodes[3 * id[0] + 2]);
        const V3<double> p1 = mk(nodes[3 * id[1]], nodes[3 * id[1] + 1], nodes[3 * id[1] + 2]);
        const V3<double> p2 = mk(nodes[3 * id[2]], nodes[3 * id[2] + 1], nodes[3 * id[2] + 2]);
        const int io = tets[4 * t + opp];
        const V3<double> po = mk(nodes[3 * io], nodes[3 * io + 1], nodes[3 * io + 2]);
        const V3<double> e1 = mk(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z);
        const V3<double> e2 = mk(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z);
        n = mk(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
        if (n.x * (po.x - p0.x) + n.y * (po.y - p0.y) + n.z * (po.z - p0.z) > 0.0) n = mk(-n.x, -n.y, -n.z);  // outward
        const double e3 = sqrt(fmax(dot3(e1, e1), fmax(dot3(e2, e2), (p2.x - p1.x) * (p2.x - p1.x) +
                                                                        (p2.y - p1.y) * (p2.y - p1.y) +
                                                                        (p2.z - p1.z) * (p2.z - p1.z))));
        tol = 1e-9 * e3 * sqrt(dot3(n, n));
        nxf = (float)n.x;
        nyf = (float)n.y;
        nzf = (float)n.z;
        tolf = __double2float_rd(tol);  // never above tol
        const double pc[3] = {p0.x, p0.y, p0.z};
        for (int k = 0; k < 3; ++k) {
            ph[k] = (float)pc[k];
            pl[k] = (float)(pc[k] - (double)ph[k]);
        }
        const float gmax = __uint_as_float(reinterpret_cast<const unsigned *>(bpos + 2 * n_bnode)[0]);
        K = 2e-13f * (fabsf(nxf) + fabsf(nyf) + fabsf(nzf)) * gmax;
    }
    // this block's chunk of the boundary nodes
    const int64_t per = (n_bnode + gridDim.y - 1) / gridDim.y;
    const int64_t b0 = blockIdx.y * per, b1 = min(n_bnode, b0 + per);
    bool outside = false;
    for (int64_t base = b0; base < b1; base += kConvexTile) {
        const int cnt = (int)min((int64_t)kConvexTile, b1 - base);
        __syncthreads();
        for (int k = threadIdx.x; k < 2 * cnt; k += kConvexFaces) sh[k] = bpos[2 * base + k];
        __syncthreads();
        if (!active || outside) continue;
        for (int j = 0; j < cnt; ++j) {
            const float4 qh = sh[2 * j], ql = sh[2 * j + 1];
            const float dx = (qh.x - ph[0]) + (ql.x - pl[0]);
            const float dy = (qh.y - ph[1]) + (ql.y - pl[1]);
            const float dz = (qh.z - ph[2]) + (ql.z - pl[2]);
            const float sf = fmaf(nxf, dx, fmaf(nyf, dy, nzf * dz));
            const float ab = fmaf(fabsf(nxf), fabsf(dx), fmaf(fabsf(nyf), fabsf(dy), fabsf(nzf) * fabsf(dz)));
            if (sf + fmaf(1e-6f, ab, K) <= tolf) continue;  // inside beyond doubt
            const int q = bnode[base + j];
            const double s = n.x * (nodes[3 * q] - p0.x) + n.y * (nodes[3 * q + 1] - p0.y) +
                             n.z * (nodes[3 * q + 2] - p0.z);
            if (s > tol) {
                outside = true;
                break;
            }
        }
    }
    if (outside) {
        atomicMax(mode, 2);  // not convex: the walk looks for re-entries
        reinterpret_cast<int *>(wrec + t * kWalkRecVec4 + 7)[opp] = -2;
    }
}

}  // namespace

bool build_walk_mesh(const int32_t *tets_host, int64_t n_nodes, int64_t n_tets, WalkMesh &w)
{
    w = WalkMesh();
    // faces as sorted vertex triples; a face shared by two tets links them
    struct Face {
        int32_t a, b, c, slot;
    };
    // in (a, b, c, slot) order: a counting sort by the smallest vertex a (the slots ascending within each a), then
    // each a's few faces sorted by (b, c, slot)
    auto face_of = [&](int64_t slot) {
        const int64_t t = slot >> 2;
        const int i = (int)(slot & 3);
        int32_t v[3], j = 0;
        for (int k = 0; k < 4; ++k)
            if (k != i) v[j++] = tets_host[4 * t + k];
        std::sort(v, v + 3);
        return Face{v[0], v[1], v[2], (int32_t)slot};
    };
    std::vector<int64_t> a_off((size_t)n_nodes + 1, 0);
    for (int64_t s = 0; s < 4 * n_tets; ++s) ++a_off[face_of(s).a + 1];
    for (int64_t q = 0; q < n_nodes; ++q) a_off[q + 1] += a_off[q];
    std::vector<Face> f((size_t)4 * n_tets);
    {
        std::vector<int64_t> at(a_off.begin(), a_off.end() - 1);
        for (int64_t s = 0; s < 4 * n_tets; ++s) {
            const Face x = face_of(s);
            f[at[x.a]++] = x;
        }
    }
    for (int64_t q = 0; q < n_nodes; ++q)
        if (a_off[q + 1] - a_off[q] > 1)
            std::sort(f.begin() + a_off[q], f.begin() + a_off[q + 1], [](const Face &x, const Face &y) {
                return std::tie(x.b, x.c, x.slot) < std::tie(y.b, y.c, y.slot);
            });
    w.nbr.assign((size_t)4 * n_tets, -1);
    bool conforming = true;
    std::vector<char> on_boundary((size_t)n_nodes, 0);
    for (size_t i = 0; i < f.size();) {
        size_t j = i + 1;
        while (j < f.size() && f[j].a == f[i].a && f[j].b == f[i].b && f[j].c == f[i].c) ++j;
        if (j - i == 2) {
            w.nbr[f[i].slot] = f[i + 1].slot >> 2;
            w.nbr[f[i + 1].slot] = f[i].slot >> 2;
        } else if (j - i == 1) {
            w.bface.push_back(f[i].slot);
            on_boundary[f[i].a] = on_boundary[f[i].b] = on_boundary[f[i].c] = 1;
        } else {
            conforming = false;  // a face shared by more than two tets
        }
        i = j;
    }
    for (int64_t q = 0; q < n_nodes; ++q)
        if (on_boundary[q]) w.bnode.push_back((int32_t)q);
    // node -> incident (tet, vertex) as a CSR list
    w.inc_off.assign((size_t)n_nodes + 1, 0);
    for (int64_t e = 0; e < 4 * n_tets; ++e) ++w.inc_off[tets_host[e] + 1];
    for (int64_t q = 0; q < n_nodes; ++q) {
        if (w.inc_off[q + 1] == 0) conforming = false;  // a node of no tet: the walk cannot start there
        w.inc_off[q + 1] += w.inc_off[q];
    }
    w.inc.assign((size_t)4 * n_tets, 0);
    std::vector<int32_t> fill(w.inc_off.begin(), w.inc_off.end() - 1);
    for (int64_t t = 0; t < n_tets; ++t)
        for (int i = 0; i < 4; ++i) w.inc[fill[tets_host[4 * t + i]]++] = (int32_t)(4 * t + i);
    w.conforming = conforming;
    return true;
}

cudaError_t launch_convex_check(const double *nodes, const int32_t *tets, const int32_t *nbr, int64_t n_tets,
                                const int32_t *bface, int64_t n_bface, const int32_t *bnode, int64_t n_bnode,
                                float4 *bpos, int conforming, int *mode, float4 *wrec, cudaStream_t st)
{
    set_int_kernel<<<1, 1, 0, st>>>(mode, conforming ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !conforming) return e;
    if (n_tets > 0) {
        fold_kernel<<<(unsigned)((4 * n_tets + 255) / 256), 256, 0, st>>>(nodes, tets, nbr, n_tets, mode);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (n_bface == 0 || n_bnode == 0) return e;
    if ((e = cudaMemsetAsync(bpos + 2 * n_bnode, 0, sizeof(float4), st)) != cudaSuccess) return e;
    bnode_split_kernel<<<(unsigned)std::min<int64_t>((n_bnode + 255) / 256, 1024), 256, 0, st>>>(nodes, bnode, n_bnode,
                                                                                                  bpos);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // face blocks x node chunks: about 16 blocks per SM, chunks of at least one tile
    const int64_t gx = (n_bface + kConvexFaces - 1) / kConvexFaces;
    const int64_t tiles = (n_bnode + kConvexTile - 1) / kConvexTile;
    const int64_t gy = std::max<int64_t>(1, std::min<int64_t>({tiles, (2432 + gx - 1) / gx, 65535}));
    if (gx > INT32_MAX) return cudaErrorInvalidValue;
    convex_kernel<<<dim3((unsigned)gx, (unsigned)gy), kConvexFaces, 0, st>>>(nodes, tets, bface, n_bface, bnode,
                                                                             n_bnode, bpos, mode, wrec);
    return cudaGetLastError();
}

cudaError_t launch_walk_records(const float4 *near32, const int32_t *nbr, int64_t n_tets, float4 *wrec,
                                cudaStream_t st)
{
    if (n_tets == 0) return cudaSuccess;
    walk_records_kernel<<<(unsigned)((n_tets + 255) / 256), 256, 0, st>>>(near32, nbr, n_tets, wrec);
    return cudaGetLastError();
}

cudaError_t launch_walk_grid(const double *nodes, const int32_t *tets, const int32_t *bface, int64_t n_bface,
                             const int32_t *bnode, int64_t n_bnode, const WalkGridArrays &g, cudaStream_t st)
{
    if (n_bface == 0 || n_bnode == 0) return cudaSuccess;
    const int64_t cells = (int64_t)g.G * g.G * g.G;
    grid_box_kernel<<<1, 256, 0, st>>>(nodes, bnode, n_bnode, g.G, g.grid);
    cudaError_t e = cudaMemsetAsync(g.cell_cnt, 0, sizeof(int32_t) * cells, st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((n_bface + 127) / 128);
    grid_faces_kernel<0><<<blocks, 128, 0, st>>>(nodes, tets, bface, n_bface, g.grid, g.cell_cnt, g.cell_off,
                                                 g.cell_face, g.cap, g.geo, g.geo32);
    grid_scan_kernel<<<1, 1024, 0, st>>>(g.cell_cnt, (int)cells, g.cell_off, g.cap, g.grid);
    if ((e = cudaMemsetAsync(g.cell_cnt, 0, sizeof(int32_t) * cells, st)) != cudaSuccess) return e;
    grid_faces_kernel<1><<<blocks, 128, 0, st>>>(nodes, tets, bface, n_bface, g.grid, g.cell_cnt, g.cell_off,
                                                 g.cell_face, g.cap, g.geo, g.geo32);
    return cudaGetLastError();
}

cudaError_t launch_walk_finalize(const WalkGrid *g, int *mode, cudaStream_t st)
{
    grid_finalize_kernel<<<1, 1, 0, st>>>(g, mode);
    return cudaGetLastError();
}

namespace {
// max over tets of (far_ratio rho + Rb) as float bits (positive floats order as their bit patterns)
__global__ void near_reach_kernel(const double *__restrict__ rho2, const double *__restrict__ near64, int64_t n_tets,
                                  double far_ratio, unsigned *bits)
{
    float m = 0.f;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tets; t += (int64_t)gridDim.x * blockDim.x) {
        const double reach = (far_ratio * sqrt(rho2[t]) + sqrt(near64[t * kNearF64 + nf64::RB2])) * (1.0 + 1e-4);
        m = fmaxf(m, __double2float_ru(reach));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(bits, __float_as_uint(m));
}
}  // namespace

cudaError_t launch_near_reach(const double *rho2, const double *near64, int64_t n_tets, double far_ratio,
                              float *r_stop, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(r_stop, 0, sizeof(float), st);
    if (e != cudaSuccess || n_tets == 0) return e;
    const int64_t blocks = std::min<int64_t>((n_tets + 255) / 256, 4096);
    near_reach_kernel<<<(unsigned)blocks, 256, 0, st>>>(rho2, near64, n_tets, far_ratio,
                                                        reinterpret_cast<unsigned *>(r_stop));
    return cudaGetLastError();
}

cudaError_t launch_walk(int precision, const WalkArgs &a, cudaStream_t st, cudaEvent_t ev_start, cudaEvent_t ev_stop)
{
    cudaError_t e;
    if (ev_start && (e = cudaEventRecord(ev_start, st)) != cudaSuccess) return e;
    const int64_t blocks = (a.n_nodes + kWalkThreads / 32 - 1) / (kWalkThreads / 32);
    // the convex-domain instance and the one with re-entries (only the one the mode selects does any work)
#define BS_WALK_PAIR(T_, G_)                                                          \
    walk_kernel<T_, G_, false, false><<<(unsigned)blocks, kWalkThreads, 0, st>>>(a);  \
    walk_kernel<T_, G_, true, false><<<(unsigned)blocks, kWalkThreads, 0, st>>>(a)
    if (a.near_mode) {
        if (a.dout || !a.perm || !a.near_out || !a.far || !a.tile_hdr || !a.r_stop || a.tile <= 0)
            return cudaErrorInvalidValue;
        if (precision == BS_FP32) {
            walk_kernel<float, false, false, true><<<(unsigned)blocks, kWalkThreads, 0, st>>>(a);
            walk_kernel<float, false, true, true><<<(unsigned)blocks, kWalkThreads, 0, st>>>(a);
        } else {
            walk_kernel<double, false, false, true><<<(unsigned)blocks, kWalkThreads, 0, st>>>(a);
            walk_kernel<double, false, true, true><<<(unsigned)blocks, kWalkThreads, 0, st>>>(a);
        }
    } else if (a.dout) {
        if (precision == BS_FP32) { BS_WALK_PAIR(float, true); }
        else { BS_WALK_PAIR(double, true); }
    } else {
        if (precision == BS_FP32) { BS_WALK_PAIR(float, false); }
        else { BS_WALK_PAIR(double, false); }
    }
#undef BS_WALK_PAIR
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev_stop) e = cudaEventRecord(ev_stop, st);
    return e;
}

}  // namespace bs
