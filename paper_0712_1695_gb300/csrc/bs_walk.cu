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
// of omega along the half-line in direction d, J = I(s) - I(-s).  That holds when every line
// leaves the mesh once, i.e. on a convex domain: the library checks, after every change of
// the node positions, that every boundary node lies on the inner side of every boundary
// face's plane, and uses the walk only then (and only on a conforming mesh whose nodes all
// belong to some tet); otherwise the all-ray kernel evaluates the nodes.  The two paths are
// both queued and each returns at once when the other one is in charge, so nothing waits
// on the host.
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

// The integral of omega along one half-line x + t d, t > 0, walking the tets from node `node`.
// float32: the point as float splits (xh, xm); records from near32.
__device__ V3<float> walk_f32(const WalkArgs &a, int64_t node, const float xh[3], const float xm[3], V3<float> d,
                              int &hits)
{
    V3<float> I = mk(0.f, 0.f, 0.f);
    // start tet: the incident tet whose face planes through x the half-line enters (largest margin)
    int T = -1, kk = -1;
    float best = -INFINITY;
    for (int e = a.inc_off[node]; e < a.inc_off[node + 1]; ++e) {
        const int code = a.inc[e];
        const int t = code >> 2, k = code & 3;
        const float4 *r = a.wrec + (int64_t)t * kWalkRecVec4;
        const float4 q0 = __ldg(r), q1 = __ldg(r + 1), q2 = __ldg(r + 2);
        const V3<float> g1 = mk(q0.x, q0.y, q0.z), g2 = mk(q1.x, q1.y, q1.z), g3 = mk(q2.x, q2.y, q2.z);
        const V3<float> g0 = mk(-(g1.x + g2.x + g3.x), -(g1.y + g2.y + g3.y), -(g1.z + g2.z + g3.z));
        float m = INFINITY;
        if (k != 0) m = fminf(m, dot3(g0, d) * rsqrtf(dot3(g0, g0)));
        if (k != 1) m = fminf(m, dot3(g1, d) * rsqrtf(dot3(g1, g1)));
        if (k != 2) m = fminf(m, dot3(g2, d) * rsqrtf(dot3(g2, g2)));
        if (k != 3) m = fminf(m, dot3(g3, d) * rsqrtf(dot3(g3, g3)));
        if (m > best) {
            best = m;
            T = t;
            kk = k;
        }
    }
    if (T < 0 || best < -kStartTolF) return I;  // the half-line leaves the mesh at x
    for (int step = 0; T >= 0; ++step) {
        if (step >= a.max_steps) {
            atomicOr(a.flag, kFlagWalk);
            break;
        }
        const float4 *r = a.wrec + (int64_t)T * kWalkRecVec4;
        const float4 q0 = __ldg(r), q1 = __ldg(r + 1), q2 = __ldg(r + 2), q3 = __ldg(r + 3);
        V3<float> g[4];
        g[1] = mk(q0.x, q0.y, q0.z);
        g[2] = mk(q1.x, q1.y, q1.z);
        g[3] = mk(q2.x, q2.y, q2.z);
        g[0] = mk(-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z));
        float av[4];
        if (step == 0) {
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
        float lo = -INFINITY, hi = INFINITY;
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
                } else if (ti < hi) {
                    hi = ti;
                    exitf = i;
                }
            }
        }
        if (exitf < 0) {  // no face ahead: not a bounded tet along this line
            atomicOr(a.flag, kFlagWalk);
            break;
        }
        // omega at the vertices (w0 w1 w2 w3, 12 floats) and the face neighbours (4 ints)
        const float4 q4 = __ldg(r + 4), q5 = __ldg(r + 5), q6 = __ldg(r + 6);
        const int4 nb = __ldg(reinterpret_cast<const int4 *>(r + 7));
        if (!empty && hi - lo > (float)kTau * q0.w) {
            const float l0 = fmaxf(lo, 0.f);
            const float f1 = hi - l0, f2 = 0.5f * (hi * hi - l0 * l0);
            const float c0 = f1 * av[0] + f2 * b[0], c1 = f1 * av[1] + f2 * b[1];
            const float c2 = f1 * av[2] + f2 * b[2], c3 = f1 * av[3] + f2 * b[3];
            I.x += c0 * q4.x + c1 * q4.w + c2 * q5.z + c3 * q6.y;
            I.y += c0 * q4.y + c1 * q5.x + c2 * q5.w + c3 * q6.z;
            I.z += c0 * q4.z + c1 * q5.y + c2 * q6.x + c3 * q6.w;
            ++hits;
        }
        T = exitf == 0 ? nb.x : exitf == 1 ? nb.y : exitf == 2 ? nb.z : nb.w;
    }
    return I;
}

// float64 form: records from near64.
__device__ V3<double> walk_f64(const WalkArgs &a, int64_t node, V3<double> x, V3<double> d, int &hits)
{
    V3<double> I = mk(0.0, 0.0, 0.0);
    int T = -1, kk = -1;
    double best = -INFINITY;
    for (int e = a.inc_off[node]; e < a.inc_off[node + 1]; ++e) {
        const int code = a.inc[e];
        const int t = code >> 2, k = code & 3;
        const double *r = a.near64 + (int64_t)t * kNearF64;
        V3<double> g[4];
        for (int i = 1; i < 4; ++i) g[i] = mk(r[nf64::G + 3 * i - 3], r[nf64::G + 3 * i - 2], r[nf64::G + 3 * i - 1]);
        g[0] = mk(-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z));
        double m = INFINITY;
        for (int i = 0; i < 4; ++i)
            if (i != k) m = fmin(m, dot3(g[i], d) / sqrt(dot3(g[i], g[i])));
        if (m > best) {
            best = m;
            T = t;
            kk = k;
        }
    }
    if (T < 0 || best < -kStartTolD) return I;
    for (int step = 0; T >= 0; ++step) {
        if (step >= a.max_steps) {
            atomicOr(a.flag, kFlagWalk);
            break;
        }
        const double *r = a.near64 + (int64_t)T * kNearF64;
        V3<double> g[4];
        for (int i = 1; i < 4; ++i) g[i] = mk(r[nf64::G + 3 * i - 3], r[nf64::G + 3 * i - 2], r[nf64::G + 3 * i - 1]);
        g[0] = mk(-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z));
        double av[4];
        if (step == 0) {
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
        double lo = -INFINITY, hi = INFINITY;
        int exitf = -1;
        bool empty = false;
        for (int i = 0; i < 4; ++i) {
            if (b[i] * b[i] <= kParD * kParD * dot3(g[i], g[i])) {
                empty = empty || (av[i] < -kParD);
            } else {
                const double ti = -av[i] / b[i];
                if (b[i] > 0.0) {
                    lo = fmax(lo, ti);
                } else if (ti < hi) {
                    hi = ti;
                    exitf = i;
                }
            }
        }
        if (exitf < 0) {
            atomicOr(a.flag, kFlagWalk);
            break;
        }
        if (!empty && hi - lo > kTau * r[nf64::H]) {
            const double l0 = fmax(lo, 0.0);
            const double f1 = hi - l0, f2 = 0.5 * (hi * hi - l0 * l0);
            for (int i = 0; i < 4; ++i) {
                const double c = f1 * av[i] + f2 * b[i];
                I.x += c * r[nf64::W + 3 * i];
                I.y += c * r[nf64::W + 3 * i + 1];
                I.z += c * r[nf64::W + 3 * i + 2];
            }
            ++hits;
        }
        T = a.nbr[4 * (int64_t)T + exitf];
    }
    return I;
}

template <typename T>
__global__ void __launch_bounds__(kWalkThreads) walk_kernel(const WalkArgs a)
{
    if (!*a.mode) return;  // not a convex conforming mesh: the all-ray kernel takes the nodes
    const int lane = threadIdx.x & 31;
    const int64_t node = (int64_t)blockIdx.x * (kWalkThreads / 32) + (threadIdx.x >> 5);
    if (node >= a.n_nodes) return;  // whole warps
    const V3<double> xd = mk(a.nodes[3 * node], a.nodes[3 * node + 1], a.nodes[3 * node + 2]);
    T ax = 0, ay = 0, az = 0;
    int hits = 0;
    if constexpr (sizeof(T) == 4) {
        float xh[3], xm[3], xl;
        split3(xd.x, xh[0], xm[0], xl);
        split3(xd.y, xh[1], xm[1], xl);
        split3(xd.z, xh[2], xm[2], xl);
        for (int l = lane; l < a.L; l += 32) {
            const float4 ln = __ldg(a.lines32 + l);
            const V3<float> s = mk(ln.x, ln.y, ln.z);
            const V3<float> Ip = walk_f32(a, node, xh, xm, s, hits);
            const V3<float> Im = walk_f32(a, node, xh, xm, mk(-s.x, -s.y, -s.z), hits);
            const V3<float> J = mk(Ip.x - Im.x, Ip.y - Im.y, Ip.z - Im.z);
            ax += ln.w * (s.y * J.z - s.z * J.y);
            ay += ln.w * (s.z * J.x - s.x * J.z);
            az += ln.w * (s.x * J.y - s.y * J.x);
        }
    } else {
        for (int l = lane; l < a.L; l += 32) {
            const dbl4 ln = a.lines64[l];
            const V3<double> s = mk(ln.x, ln.y, ln.z);
            const V3<double> Ip = walk_f64(a, node, xd, s, hits);
            const V3<double> Im = walk_f64(a, node, xd, mk(-s.x, -s.y, -s.z), hits);
            const V3<double> J = mk(Ip.x - Im.x, Ip.y - Im.y, Ip.z - Im.z);
            ax += ln.w * (s.y * J.z - s.z * J.y);
            ay += ln.w * (s.z * J.x - s.x * J.z);
            az += ln.w * (s.x * J.y - s.y * J.x);
        }
    }
    ax = warp_sum(ax);
    ay = warp_sum(ay);
    az = warp_sum(az);
    hits = warp_sum(hits);
    if (lane == 0) {
        a.out[3 * node] = (double)ax;
        a.out[3 * node + 1] = (double)ay;
        a.out[3 * node + 2] = (double)az;
        if (a.counts) {
            a.counts[3 * node] = (int32_t)min(a.n_tets, (int64_t)INT32_MAX);
            a.counts[3 * node + 1] = 0;
            a.counts[3 * node + 2] = hits;
        }
    }
}

__global__ void set_int_kernel(int *p, int v) { *p = v; }

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
__global__ void convex_kernel(const double *__restrict__ nodes, const int32_t *__restrict__ tets,
                              const int32_t *__restrict__ bface, int64_t n_bface, const int32_t *__restrict__ bnode,
                              int64_t n_bnode, int *mode)
{
    const int64_t f = blockIdx.y;  // boundary face of this block row
    if (f >= n_bface || !*mode) return;
    const int slot = bface[f];
    const int64_t t = slot >> 2;
    const int opp = slot & 3;
    int id[3], j = 0;
    for (int i = 0; i < 4; ++i)
        if (i != opp) id[j++] = tets[4 * t + i];
    const V3<double> p0 = mk(nodes[3 * id[0]], nodes[3 * id[0] + 1], nodes[3 * id[0] + 2]);
    const V3<double> p1 = mk(nodes[3 * id[1]], nodes[3 * id[1] + 1], nodes[3 * id[1] + 2]);
    const V3<double> p2 = mk(nodes[3 * id[2]], nodes[3 * id[2] + 1], nodes[3 * id[2] + 2]);
    const int io = tets[4 * t + opp];
    const V3<double> po = mk(nodes[3 * io], nodes[3 * io + 1], nodes[3 * io + 2]);
    const V3<double> e1 = mk(p1.x - p0.x, p1.y - p0.y, p1.z - p0.z), e2 = mk(p2.x - p0.x, p2.y - p0.y, p2.z - p0.z);
    V3<double> n = mk(e1.y * e2.z - e1.z * e2.y, e1.z * e2.x - e1.x * e2.z, e1.x * e2.y - e1.y * e2.x);
    if (n.x * (po.x - p0.x) + n.y * (po.y - p0.y) + n.z * (po.z - p0.z) > 0.0) n = mk(-n.x, -n.y, -n.z);  // outward
    const double e3 = sqrt(fmax(dot3(e1, e1), fmax(dot3(e2, e2), (p2.x - p1.x) * (p2.x - p1.x) +
                                                                    (p2.y - p1.y) * (p2.y - p1.y) +
                                                                    (p2.z - p1.z) * (p2.z - p1.z))));
    const double tol = 1e-9 * e3 * sqrt(dot3(n, n));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_bnode; i += (int64_t)gridDim.x * blockDim.x) {
        const int q = bnode[i];
        const double s = n.x * (nodes[3 * q] - p0.x) + n.y * (nodes[3 * q + 1] - p0.y) + n.z * (nodes[3 * q + 2] - p0.z);
        if (s > tol) {
            atomicAnd(mode, 0);
            return;
        }
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
    std::vector<Face> f((size_t)4 * n_tets);
    for (int64_t t = 0; t < n_tets; ++t)
        for (int i = 0; i < 4; ++i) {
            int32_t v[3], j = 0;
            for (int k = 0; k < 4; ++k)
                if (k != i) v[j++] = tets_host[4 * t + k];
            std::sort(v, v + 3);
            f[4 * t + i] = {v[0], v[1], v[2], (int32_t)(4 * t + i)};
        }
    std::sort(f.begin(), f.end(), [](const Face &x, const Face &y) {
        return std::tie(x.a, x.b, x.c, x.slot) < std::tie(y.a, y.b, y.c, y.slot);
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

cudaError_t launch_convex_check(const double *nodes, const int32_t *tets, const int32_t *bface, int64_t n_bface,
                                const int32_t *bnode, int64_t n_bnode, int conforming, int *mode, cudaStream_t st)
{
    set_int_kernel<<<1, 1, 0, st>>>(mode, conforming ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !conforming || n_bface == 0 || n_bnode == 0) return e;
    const int64_t gx = std::min<int64_t>((n_bnode + 255) / 256, 8);
    for (int64_t f0 = 0; f0 < n_bface; f0 += 65535) {
        const dim3 grid((unsigned)gx, (unsigned)std::min<int64_t>(65535, n_bface - f0));
        convex_kernel<<<grid, 256, 0, st>>>(nodes, tets, bface + f0, n_bface - f0, bnode, n_bnode, mode);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_walk_records(const float4 *near32, const int32_t *nbr, int64_t n_tets, float4 *wrec,
                                cudaStream_t st)
{
    if (n_tets == 0) return cudaSuccess;
    walk_records_kernel<<<(unsigned)((n_tets + 255) / 256), 256, 0, st>>>(near32, nbr, n_tets, wrec);
    return cudaGetLastError();
}

cudaError_t launch_walk(int precision, const WalkArgs &a, cudaStream_t st, cudaEvent_t ev_start, cudaEvent_t ev_stop)
{
    cudaError_t e;
    if (ev_start && (e = cudaEventRecord(ev_start, st)) != cudaSuccess) return e;
    const int64_t blocks = (a.n_nodes + kWalkThreads / 32 - 1) / (kWalkThreads / 32);
    if (precision == BS_FP32) walk_kernel<float><<<(unsigned)blocks, kWalkThreads, 0, st>>>(a);
    else walk_kernel<double><<<(unsigned)blocks, kWalkThreads, 0, st>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev_stop) e = cudaEventRecord(ev_stop, st);
    return e;
}

}  // namespace bs
