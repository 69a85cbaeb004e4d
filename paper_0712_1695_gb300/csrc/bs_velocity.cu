// bs_velocity.cu -- selection and launch of the velocity kernel's variants (instantiated in the
// bs_vel_*.cu files from bs_velocity_kernel.cuh), the deterministic reduction of the per-chunk partial
// sums, and the launch helpers the C ABI uses.
#include <math.h>

#include <algorithm>

#include "bs_near_pass.cuh"
#include "bs_velocity_kernel.cuh"

namespace bs {
namespace {

// out[perm[i]] = sum over chunks of partial[chunk][i] (fixed chunk order);
// batch: one thread per point of all meshes, the mesh found from point_begin.
__global__ void reduce_kernel(const VelocityArgs a)
{
    if (a.skip && *a.skip) return;  // the mesh walk wrote the output
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const MeshDesc *m = &a.m;
    int64_t i = g;
    if (a.meshes) {
        if (g >= a.n_points) return;
        int lo = 0, hi = a.n_meshes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.meshes[mid].point_begin <= g) lo = mid;
            else hi = mid - 1;
        }
        m = &a.meshes[lo];
        i = g - m->point_begin;
    }
    const int64_t k = m->k;
    if (i >= k) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int c = 0; c < m->n_chunks; ++c) {
        const double *q = m->partial + (c * k + i) * 3;
        s0 += q[0];
        s1 += q[1];
        s2 += q[2];
    }
    if (a.near_out && m->n_tets > 0) {  // the near pass's totals, its parts in order
        const int split = a.meshes ? 1 : max(a.near_split, 1);
        for (int s = 0; s < split; ++s) {
            const double *q = a.near_out + s * a.near_split_stride + 3 * ((a.meshes ? m->point_begin : 0) + i);
            s0 += q[0];
            s1 += q[1];
            s2 += q[2];
        }
    }
    const int64_t o = m->perm[i];
    m->out[3 * o + 0] = s0;
    m->out[3 * o + 1] = s1;
    m->out[3 * o + 2] = s2;
}

__global__ void zero_kernel(int32_t *counts, int64_t n, unsigned long long *work_counter, const int *skip)
{
    if (skip && *skip) return;  // the mesh walk evaluated these points
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0) *work_counter = 0ull;
    if (counts && i < n) counts[i] = 0;
}

}  // namespace

VariantList velocity_variants(int precision, int Q, int near_rule)
{
    if (near_rule == BS_NEAR_EXACT) return variants_exact(precision, Q);
    if (precision == BS_FP64) return variants_f64(Q);
    return Q == 4 ? variants_f32_q4() : variants_f32_rules(Q);
}

int num_variants(int precision, int Q, int near_rule) { return velocity_variants(precision, Q, near_rule).n; }

int small_mesh_variant(int precision, int Q, bool near_pass)
{
    if (precision != BS_FP32 || Q != 4) return -1;
    const VariantList vl = velocity_variants(precision, Q, BS_NEAR_RAY);
    for (int v = 0; v < vl.n; ++v) {
        const VariantShape &s = vl.v[v].s;
        if (s.P == 1 && s.U == 1 && s.TILE == 32 && !s.PK && (s.DR == 3) == near_pass) return v;
    }
    return -1;
}

int near_pass_variant(int precision, int Q, int near_rule)
{
    const VariantList vl = velocity_variants(precision, Q, near_rule);
    for (int v = 0; v < vl.n; ++v)
        if (vl.v[v].s.DR == 3) return v;
    return -1;
}

int noalloc_variant(int precision, int Q, int near_rule)
{
    const VariantList vl = velocity_variants(precision, Q, near_rule);
    int best = -1;
    for (int v = 0; v < vl.n; ++v) {
        const VariantShape &s = vl.v[v].s;
        if (s.PK || s.TILE > 32 || s.TILE < 8 || s.DR == 3) continue;
        if (best < 0 || (near_rule == BS_NEAR_RAY && s.P == 1 && vl.v[best].s.P != 1)) best = v;
    }
    return best;
}

LaunchShape shape_for(int precision, int Q, int variant, int near_rule)
{
    const VariantList vl = velocity_variants(precision, Q, near_rule);
    LaunchShape s;
    if (vl.n == 0) return s;
    const VariantShape &v = vl.v[(variant >= 0 && variant < vl.n) ? variant : 0].s;
    s.threads = 128;
    s.points_per_thread = v.P;
    s.tile = v.TILE;
    s.layout = v.PK ? kFarPointPairs : kFarQuadPairs;
    s.drain = v.DR;
    return s;
}

int velocity_ctas_per_sm(int precision, int Q, int variant, int near_rule)
{
    const VariantList vl = velocity_variants(precision, Q, near_rule);
    if (vl.n == 0) return 0;
    VelocityArgs q;
    q.Q = Q;
    q.variant = variant;
    q.near_rule = near_rule;
    int occ = 0;
    if (vl.v[(variant >= 0 && variant < vl.n) ? variant : 0].launch(q, 1, 0, nullptr, true, &occ) != cudaSuccess)
        return 0;
    return occ;
}

cudaError_t launch_velocity(int precision, const VelocityArgs &a, int n_sm, cudaStream_t st, int *grid_out,
                            cudaEvent_t ev_start, cudaEvent_t ev_stop)
{
    const VariantList vl = velocity_variants(precision, a.Q, a.near_rule);
    if (vl.n == 0 || a.variant < 0 || a.variant >= vl.n) return cudaErrorInvalidValue;
    const int64_t nc = a.counts ? 3 * a.m.k : 0;
    zero_kernel<<<(unsigned)((nc + 255) / 256 + 1), 256, 0, st>>>(a.counts, nc, a.work_counter, a.skip);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev_start && (e = cudaEventRecord(ev_start, st)) != cudaSuccess) return e;
    e = vl.v[a.variant].launch(a, n_sm, st, grid_out, false, nullptr);
    if (e != cudaSuccess) return e;
    if (ev_stop) e = cudaEventRecord(ev_stop, st);
    return e;
}

cudaError_t launch_near_pass(int precision, const VelocityArgs &a, cudaStream_t st)
{
    const VariantList vl = velocity_variants(precision, a.Q, a.near_rule);
    if (vl.n == 0 || a.variant < 0 || a.variant >= vl.n) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (vl.v[a.variant].s.DR == 3 && a.n_near_warps > 0) {
        if (!a.near_out || a.tile <= 0 || a.far_stride <= 0) return cudaErrorInvalidValue;
        const size_t sm = a.smem_lines ? sizeof(float4) * a.L : 0;
        const int split = a.meshes ? 1 : std::max(a.near_split, 1);
        if (a.n_near_warps * split > INT32_MAX) return cudaErrorInvalidValue;
        const unsigned blocks = (unsigned)(a.n_near_warps * split);  // one CTA per (32 points, part of the tiles)
        auto go = [&](auto kern, int nw) -> cudaError_t {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (r != cudaSuccess) return r;
            kern<<<blocks, 32 * nw, sm, st>>>(a);
            return cudaGetLastError();
        };
        if (precision == BS_FP32)
            e = go(near_pass_kernel<float, kNearPassWarps>, kNearPassWarps);
        else
            e = go(near_pass_kernel<double, kNearPassWarps>, kNearPassWarps);
    }
    return e;
}

cudaError_t launch_reduce(const VelocityArgs &a, cudaStream_t st)
{
    const int64_t n = a.meshes ? a.n_points : a.m.k;
    reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace bs
