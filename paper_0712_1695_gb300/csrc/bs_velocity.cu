// bs_velocity.cu -- velocity at evaluation points (Eq. 1 by the far tet rule
// and the ray rule of Section 2), float32 and float64 variants.
//
// Work decomposition (N-body style, one GPU):
//   item = (block of P*NT evaluation points, chunk of consecutive tet tiles).
//   A persistent grid pulls items from a device counter.  Each CTA keeps its
//   points in registers (P per thread) and in shared memory, and streams the
//   chunk's far records tile by tile into a double-buffered shared-memory
//   ring with one bulk asynchronous copy (cp.async.bulk + mbarrier) per tile.
//   Every thread classifies its points against each tet of the tile (one
//   warp-uniform broadcast read of the record per tet); far pairs go through
//   the tet Gauss rule, near pairs are appended to a per-warp queue with a
//   warp ballot.  The queue is drained by the whole warp: the 32 lanes split
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
#include <math.h>

#include <algorithm>

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
constexpr long long kWaitCap = 1LL << 26;

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
// bounded wait: false when the cap is reached
__device__ inline bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (long long i = 0; i < kWaitCap; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
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
__device__ inline T inv_sqrt(T r2);
template <>
__device__ inline float inv_sqrt<float>(float r2) { return rsqrtf(r2); }
template <>
__device__ inline double inv_sqrt<double>(double r2) { return 1.0 / sqrt(r2); }

template <typename T>
__device__ inline T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Ray rule for one (point, tet) pair, lines split across the 32 lanes.
// Returns the warp-reduced contribution (all lanes) and the hit count.
// ---------------------------------------------------------------------------
struct NearOut {
    double vx, vy, vz;
    int hits;
};

// float64 version: every step in double.  Used by the float64 path and by
// degenerate pairs of the float32 path.
__device__ __noinline__ NearOut near_pair_f64(V3<double> x, const double *__restrict__ r, const dbl4 *__restrict__ lines,
                                 int L, int lane)
{
    V3<double> v[4];
    int vk = -1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        v[i] = mk(r[nf64::V + 3 * i], r[nf64::V + 3 * i + 1], r[nf64::V + 3 * i + 2]);
        if (vk < 0 && v[i].x == x.x && v[i].y == x.y && v[i].z == x.z) vk = i;
    }
    const V3<double> g1 = mk(r[nf64::G + 0], r[nf64::G + 1], r[nf64::G + 2]);
    const V3<double> g2 = mk(r[nf64::G + 3], r[nf64::G + 4], r[nf64::G + 5]);
    const V3<double> g3 = mk(r[nf64::G + 6], r[nf64::G + 7], r[nf64::G + 8]);
    V3<double> w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = mk(r[nf64::W + 3 * i], r[nf64::W + 3 * i + 1], r[nf64::W + 3 * i + 2]);
    const double h = r[nf64::H], rb2 = r[nf64::RB2];
    const V3<double> d0 = mk(x.x - v[0].x, x.y - v[0].y, x.z - v[0].z);
    double a[4];
    if (vk >= 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = (i == vk) ? 1.0 : 0.0;
    } else {
        a[1] = dot3(g1, d0);
        a[2] = dot3(g2, d0);
        a[3] = dot3(g3, d0);
        a[0] = 1.0 - a[1] - a[2] - a[3];
    }
    const V3<double> Wa = mk(a[0] * w[0].x + a[1] * w[1].x + a[2] * w[2].x + a[3] * w[3].x,
                             a[0] * w[0].y + a[1] * w[1].y + a[2] * w[2].y + a[3] * w[3].y,
                             a[0] * w[0].z + a[1] * w[1].z + a[2] * w[2].z + a[3] * w[3].z);
    const V3<double> rc = mk(r[nf64::C] - x.x, r[nf64::C + 1] - x.y, r[nf64::C + 2] - x.z);
    const double rc2 = dot3(rc, rc);
    const double bound = rb2 * (1.0 + kBoundPadD);
    const V3<double> g0 = mk(-(g1.x + g2.x + g3.x), -(g1.y + g2.y + g3.y), -(g1.z + g2.z + g3.z));
    const double par2[4] = {kParD * kParD * dot3(g0, g0), kParD * kParD * dot3(g1, g1),
                            kParD * kParD * dot3(g2, g2), kParD * kParD * dot3(g3, g3)};
    double ax = 0.0, ay = 0.0, az = 0.0;
    int hits = 0;
    for (int l = lane; l < L; l += 32) {
        const dbl4 ln = lines[l];
        const V3<double> s = mk(ln.x, ln.y, ln.z);
        const double rs = dot3(rc, s);
        if (rc2 - rs * rs > bound) continue;  // line farther than Rb from the centroid
        double b[4];
        b[1] = dot3(g1, s);
        b[2] = dot3(g2, s);
        b[3] = dot3(g3, s);
        b[0] = -(b[1] + b[2] + b[3]);
        double lo = -INFINITY, hi = INFINITY;
        bool empty = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (b[i] * b[i] <= par2[i]) empty = empty || (a[i] < -kParD);
            else if (b[i] > 0.0) lo = fmax(lo, -a[i] / b[i]);
            else hi = fmin(hi, -a[i] / b[i]);
        }
        if (empty || !(hi - lo > kTau * h)) continue;
        const V3<double> Wb = mk(b[0] * w[0].x + b[1] * w[1].x + b[2] * w[2].x + b[3] * w[3].x,
                                 b[0] * w[0].y + b[1] * w[1].y + b[2] * w[2].y + b[3] * w[3].y,
                                 b[0] * w[0].z + b[1] * w[1].z + b[2] * w[2].z + b[3] * w[3].z);
        const double f1 = fabs(hi) - fabs(lo);
        const double f2 = 0.5 * (hi * fabs(hi) - lo * fabs(lo));
        const V3<double> J = mk(f1 * Wa.x + f2 * Wb.x, f1 * Wa.y + f2 * Wb.y, f1 * Wa.z + f2 * Wb.z);
        ax += ln.w * (s.y * J.z - s.z * J.y);
        ay += ln.w * (s.z * J.x - s.x * J.z);
        az += ln.w * (s.x * J.y - s.y * J.x);
        ++hits;
    }
    NearOut o;
    o.vx = warp_sum(ax);
    o.vy = warp_sum(ay);
    o.vz = warp_sum(az);
    o.hits = warp_sum(hits);
    return o;
}

// float32 version.  The differences x - v0 and c - x are taken in float64
// and rounded once, so a_i carries no error from the absolute coordinates.
// Pairs whose point is on (or within 1e-5 in barycentric units of) the
// boundary of the tet go to the float64 version: there the chord can jump
// with the sign of a tiny b_i and float32 rounding would pick a side at
// random.
__device__ __noinline__ NearOut near_pair_f32(V3<double> x, const float4 *__restrict__ r32, const double *__restrict__ r64,
                                 const float4 *__restrict__ lines, const dbl4 *__restrict__ lines64, int L,
                                 int lane)
{
    const V3<double> v0 = mk(r64[nf64::V], r64[nf64::V + 1], r64[nf64::V + 2]);
    bool at_vertex = false;
#pragma unroll
    for (int i = 0; i < 4; ++i)
        at_vertex = at_vertex || (r64[nf64::V + 3 * i] == x.x && r64[nf64::V + 3 * i + 1] == x.y &&
                                  r64[nf64::V + 3 * i + 2] == x.z);
    const float4 q0 = r32[0], q1 = r32[1], q2 = r32[2];
    const V3<float> g1 = mk(q0.x, q0.y, q0.z), g2 = mk(q1.x, q1.y, q1.z), g3 = mk(q2.x, q2.y, q2.z);
    const float h = q0.w, rb2 = q1.w;
    const V3<float> d0 = mk((float)(x.x - v0.x), (float)(x.y - v0.y), (float)(x.z - v0.z));
    float a[4];
    a[1] = dot3(g1, d0);
    a[2] = dot3(g2, d0);
    a[3] = dot3(g3, d0);
    a[0] = 1.0f - a[1] - a[2] - a[3];
    const float amin = fminf(fminf(a[0], a[1]), fminf(a[2], a[3]));
    const float aabs = fminf(fminf(fabsf(a[0]), fabsf(a[1])), fminf(fabsf(a[2]), fabsf(a[3])));
    if (at_vertex || (amin > -kDegenA && aabs < kDegenA)) return near_pair_f64(x, r64, lines64, L, lane);

    V3<float> w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 t = r32[3 + i];
        w[i] = mk(t.x, t.y, t.z);
    }
    const V3<float> Wa = mk(a[0] * w[0].x + a[1] * w[1].x + a[2] * w[2].x + a[3] * w[3].x,
                            a[0] * w[0].y + a[1] * w[1].y + a[2] * w[2].y + a[3] * w[3].y,
                            a[0] * w[0].z + a[1] * w[1].z + a[2] * w[2].z + a[3] * w[3].z);
    const V3<float> rc = mk((float)(r64[nf64::C] - x.x), (float)(r64[nf64::C + 1] - x.y),
                            (float)(r64[nf64::C + 2] - x.z));
    const float rc2 = dot3(rc, rc);
    const float bound = rb2 * (1.0f + kBoundPadF);
    const V3<float> g0 = mk(-(g1.x + g2.x + g3.x), -(g1.y + g2.y + g3.y), -(g1.z + g2.z + g3.z));
    const float par2[4] = {kParF * kParF * dot3(g0, g0), kParF * kParF * dot3(g1, g1), kParF * kParF * dot3(g2, g2),
                           kParF * kParF * dot3(g3, g3)};
    const float tau_h = (float)kTau * h;
    float ax = 0.f, ay = 0.f, az = 0.f;
    int hits = 0;
    for (int l = lane; l < L; l += 32) {
        const float4 ln = lines[l];
        const V3<float> s = mk(ln.x, ln.y, ln.z);
        const float rs = dot3(rc, s);
        if (rc2 - rs * rs > bound) continue;
        float b[4];
        b[1] = dot3(g1, s);
        b[2] = dot3(g2, s);
        b[3] = dot3(g3, s);
        b[0] = -(b[1] + b[2] + b[3]);
        float lo = -INFINITY, hi = INFINITY;
        bool empty = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (b[i] * b[i] <= par2[i]) empty = empty || (a[i] < -kParF);
            else if (b[i] > 0.f) lo = fmaxf(lo, -a[i] / b[i]);
            else hi = fminf(hi, -a[i] / b[i]);
        }
        if (empty || !(hi - lo > tau_h)) continue;
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
    }
    NearOut o;
    o.vx = warp_sum(ax);
    o.vy = warp_sum(ay);
    o.vz = warp_sum(az);
    o.hits = warp_sum(hits);
    return o;
}

// ---------------------------------------------------------------------------
// The velocity kernel.
// ---------------------------------------------------------------------------
template <typename T>
struct Acc;  // per-point accumulator
template <>
struct Acc<float> {
    float s[3], c[3];  // Kahan sum across tiles
};
template <>
struct Acc<double> {
    double s[3];
};

template <typename T, int Q, int P, int NT, int TILE>
__global__ void __launch_bounds__(NT) velocity_kernel(const VelocityArgs a)
{
    constexpr int RS = far_stride<T>(Q);
    constexpr int BP = NT * P;
    constexpr int NW = NT / 32;
    constexpr int QCAP = 256;
    constexpr int TILE_BYTES = TILE * RS * (int)sizeof(T);
    static_assert(TILE <= 256, "tet index in the near queue is 8 bits");
    static_assert(P * 32 <= 256, "point slot in the near queue is 8 bits");

    extern __shared__ __align__(128) unsigned char smem[];
    T *tiles = reinterpret_cast<T *>(smem);                                         // [2][TILE*RS]
    double *spts = reinterpret_cast<double *>(smem + 2 * TILE_BYTES);               // [BP][3]
    uint16_t *queue = reinterpret_cast<uint16_t *>(spts + 3 * BP);                  // [NW][QCAP]
    uint64_t *bars = reinterpret_cast<uint64_t *>(queue + NW * QCAP);               // [2]
    int *s_item = reinterpret_cast<int *>(bars + 2);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t k = a.k;
    const int64_t n_blocks = (k + BP - 1) / BP;
    const int64_t n_items = n_blocks * a.n_chunks;
    const int64_t n_tiles = (a.n_tets + TILE - 1) / TILE;
    const T fr2 = (T)a.far_ratio2;
    const T *far = reinterpret_cast<const T *>(a.far);

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase[2] = {0u, 0u};

    for (;;) {
        if (tid == 0) *s_item = atomicAdd(a.work_counter, 1);
        __syncthreads();
        const int64_t item = *s_item;
        if (item >= n_items) break;
        const int64_t pb = item % n_blocks, ck = item / n_blocks;
        const int64_t t0 = ck * a.tiles_per_chunk;
        const int64_t t1 = min(t0 + (int64_t)a.tiles_per_chunk, n_tiles);

        // kick off the first tile while the points are loaded
        auto issue = [&](int64_t t, int buf) {
            const int64_t first = t * TILE;
            const int cnt = (int)min((int64_t)TILE, a.n_tets - first);
            const uint32_t bytes = (uint32_t)cnt * RS * sizeof(T);
            mbar_expect_tx(&bars[buf], bytes);
            bulk_g2s(tiles + buf * TILE * RS, far + first * RS, bytes, &bars[buf]);
        };
        if (tid == 0 && t0 < t1) issue(t0, 0);

        for (int i = tid; i < BP; i += NT) {
            int64_t gi = pb * BP + i;
            if (gi >= k) gi = k - 1;  // pad with a real point; its result is not written
            spts[3 * i + 0] = a.pts[3 * gi + 0];
            spts[3 * i + 1] = a.pts[3 * gi + 1];
            spts[3 * i + 2] = a.pts[3 * gi + 2];
        }
        __syncthreads();

        V3<T> xp[P];
        Acc<T> acc[P];
        int nnear[P], nhit[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int slot = p * NT + tid;
            xp[p] = mk((T)spts[3 * slot], (T)spts[3 * slot + 1], (T)spts[3 * slot + 2]);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                acc[p].s[j] = 0;
                if constexpr (sizeof(T) == 4) acc[p].c[j] = 0;
            }
            nnear[p] = 0;
            nhit[p] = 0;
        }
        uint16_t *wq = queue + warp * QCAP;

        bool aborted = false;
        for (int64_t t = t0; t < t1; ++t) {
            const int buf = (int)((t - t0) & 1);
            if (tid == 0 && t + 1 < t1) issue(t + 1, buf ^ 1);
            if (!mbar_wait(&bars[buf], phase[buf])) {
                aborted = true;
                break;
            }
            phase[buf] ^= 1u;
            const T *tb = tiles + buf * TILE * RS;
            const int cnt = (int)min((int64_t)TILE, a.n_tets - t * TILE);

            T tacc[P][3];
#pragma unroll
            for (int p = 0; p < P; ++p) tacc[p][0] = tacc[p][1] = tacc[p][2] = 0;
            int qn = 0;  // warp-uniform

            auto drain = [&]() {
                for (int e = 0; e < qn; ++e) {
                    const int code = wq[e];
                    const int slot = code >> 8, j = code & 255;
                    const int pp = slot >> 5, owner = slot & 31;
                    const int bi = pp * NT + warp * 32 + owner;
                    const int64_t tet = t * TILE + j;
                    const V3<double> xd = mk(spts[3 * bi], spts[3 * bi + 1], spts[3 * bi + 2]);
                    NearOut o;
                    if constexpr (sizeof(T) == 4)
                        o = near_pair_f32(xd, a.near32 + tet * kNearF32Vec4, a.near64 + tet * kNearF64,
                                          a.lines.f32, a.lines.f64, a.L, lane);
                    else
                        o = near_pair_f64(xd, a.near64 + tet * kNearF64, a.lines.f64, a.L, lane);
                    if (lane == owner) {
#pragma unroll
                        for (int p = 0; p < P; ++p)
                            if (p == pp) {
                                tacc[p][0] += (T)o.vx;
                                tacc[p][1] += (T)o.vy;
                                tacc[p][2] += (T)o.vz;
                                nhit[p] += o.hits;
                            }
                    }
                }
                qn = 0;
                __syncwarp();
            };

            for (int j = 0; j < cnt; ++j) {
                const T *rec = tb + j * RS;
                const V3<T> c = mk(rec[0], rec[1], rec[2]);
                const T thr2 = fr2 * rec[3];
                bool nearp[P];
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const V3<T> d = mk(xp[p].x - c.x, xp[p].y - c.y, xp[p].z - c.z);
                    nearp[p] = !(dot3(d, d) > thr2);
                }
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const T *qq = rec + 4 + 6 * q;
                    const V3<T> xq = mk(qq[0], qq[1], qq[2]);
                    const V3<T> wv = mk(qq[3], qq[4], qq[5]);
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        if (nearp[p]) continue;
                        const T dx = xp[p].x - xq.x, dy = xp[p].y - xq.y, dz = xp[p].z - xq.z;
                        const T r2 = dx * dx + dy * dy + dz * dz;
                        const T ir = inv_sqrt<T>(r2);
                        const T ir3 = ir * ir * ir;
                        tacc[p][0] += ir3 * (dy * wv.z - dz * wv.y);
                        tacc[p][1] += ir3 * (dz * wv.x - dx * wv.z);
                        tacc[p][2] += ir3 * (dx * wv.y - dy * wv.x);
                    }
                }
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const unsigned m = __ballot_sync(0xffffffffu, nearp[p]);
                    if (m) {
                        if (nearp[p]) {
                            const int pos = qn + __popc(m & ((1u << lane) - 1u));
                            wq[pos] = (uint16_t)(((p * 32 + lane) << 8) | j);
                            ++nnear[p];
                        }
                        qn += __popc(m);
                    }
                }
                if (qn > QCAP - 32 * P) {
                    __syncwarp();
                    drain();
                }
            }
            if (qn > 0) {
                __syncwarp();
                drain();
            }
            // fold the tile partial into the per-point sum
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int jj = 0; jj < 3; ++jj) {
                    if constexpr (sizeof(T) == 4) {
                        const float y = tacc[p][jj] - acc[p].c[jj];
                        const float s2 = acc[p].s[jj] + y;
                        acc[p].c[jj] = (s2 - acc[p].s[jj]) - y;
                        acc[p].s[jj] = s2;
                    } else {
                        acc[p].s[jj] += tacc[p][jj];
                    }
                }
            __syncthreads();  // every warp is done with this buffer before it is refilled
        }
        if (aborted) {
            if (tid == 0) atomicOr(a.flag, kFlagTimeout);
            // let the copies still in flight land before the CTA leaves
            mbar_wait(&bars[0], phase[0]);
            mbar_wait(&bars[1], phase[1]);
            return;
        }

        const int64_t ntets_chunk = min(a.n_tets, t1 * TILE) - t0 * TILE;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int64_t gi = pb * BP + p * NT + tid;
            if (gi >= k) continue;
            double *dst = a.partial + (ck * k + gi) * 3;
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
                if constexpr (sizeof(T) == 4)
                    dst[jj] = (double)acc[p].s[jj] - (double)acc[p].c[jj];
                else
                    dst[jj] = acc[p].s[jj];
            }
            if (a.counts) {
                atomicAdd(&a.counts[3 * gi + 0], nnear[p]);
                atomicAdd(&a.counts[3 * gi + 1], (int)(ntets_chunk - nnear[p]));
                atomicAdd(&a.counts[3 * gi + 2], nhit[p]);
            }
        }
        __syncthreads();  // spts reused by the next item
    }
}

__global__ void reduce_kernel(const double *__restrict__ partial, int n_chunks, int64_t k, double *__restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * k) return;
    double s = 0.0;
    for (int c = 0; c < n_chunks; ++c) s += partial[c * 3 * k + i];
    out[i] = s;
}

__global__ void zero_kernel(int32_t *counts, int64_t n, int *work_counter)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) *work_counter = 0;
    if (counts && i < n) counts[i] = 0;
}

template <typename T, int Q, int P, int NT, int TILE>
size_t smem_bytes()
{
    constexpr int RS = far_stride<T>(Q);
    return 2 * (size_t)TILE * RS * sizeof(T) + 3 * sizeof(double) * NT * P + (NT / 32) * 256 * sizeof(uint16_t) +
           2 * sizeof(uint64_t) + 16;
}

template <typename T, int Q, int P, int NT, int TILE>
cudaError_t launch_t(const VelocityArgs &a, int n_sm, cudaStream_t st, int *grid_out, bool query_only, int *occ_out)
{
    auto kern = velocity_kernel<T, Q, P, NT, TILE>;
    const size_t sm = smem_bytes<T, Q, P, NT, TILE>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, sm);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    if (occ_out) *occ_out = occ;
    if (query_only) return cudaSuccess;
    const int64_t BP = (int64_t)NT * P;
    const int64_t n_items = ((a.k + BP - 1) / BP) * a.n_chunks;
    const int64_t grid = std::min<int64_t>(n_items, (int64_t)n_sm * occ);
    if (grid_out) *grid_out = (int)grid;
    kern<<<(unsigned)grid, NT, sm, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch(const VelocityArgs &a, int n_sm, cudaStream_t st, int *grid_out, bool qo, int *occ)
{
    switch (a.Q) {
    case 1: return launch_t<T, 1, 2, 128, 64>(a, n_sm, st, grid_out, qo, occ);
    case 4: return launch_t<T, 4, 2, 128, 64>(a, n_sm, st, grid_out, qo, occ);
    case 8: return launch_t<T, 8, 2, 128, 32>(a, n_sm, st, grid_out, qo, occ);
    case 27: return launch_t<T, 27, 1, 128, 16>(a, n_sm, st, grid_out, qo, occ);
    case 64: return launch_t<T, 64, 1, 128, 8>(a, n_sm, st, grid_out, qo, occ);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

LaunchShape shape_for(int precision, int Q)
{
    (void)precision;
    LaunchShape s;
    s.threads = 128;
    s.points_per_thread = Q <= 8 ? 2 : 1;
    s.tile = Q <= 4 ? 64 : Q == 8 ? 32 : Q == 27 ? 16 : 8;
    return s;
}

int velocity_ctas_per_sm(int precision, int Q)
{
    VelocityArgs q;
    q.Q = Q;
    int occ = 0;
    if (precision == BS_FP32)
        dispatch<float>(q, 1, 0, nullptr, true, &occ);
    else
        dispatch<double>(q, 1, 0, nullptr, true, &occ);
    return occ;
}

cudaError_t launch_velocity(int precision, const VelocityArgs &a, int n_sm, cudaStream_t st, int *grid_out,
                            cudaEvent_t ev_start, cudaEvent_t ev_stop)
{
    zero_kernel<<<(unsigned)((3 * a.k + 255) / 256 + 1), 256, 0, st>>>(a.counts, 3 * a.k, a.work_counter);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev_start && (e = cudaEventRecord(ev_start, st)) != cudaSuccess) return e;
    e = precision == BS_FP32 ? dispatch<float>(a, n_sm, st, grid_out, false, nullptr)
                             : dispatch<double>(a, n_sm, st, grid_out, false, nullptr);
    if (e != cudaSuccess) return e;
    if (ev_stop) e = cudaEventRecord(ev_stop, st);
    return e;
}

cudaError_t launch_reduce(const VelocityArgs &a, cudaStream_t st)
{
    const int64_t n = 3 * a.k;
    reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a.partial, a.n_chunks, a.k, a.out);
    return cudaGetLastError();
}

}  // namespace bs
