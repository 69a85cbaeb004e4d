// bs_near_pass.cuh -- the near pass: the near pairs a far-sweep variant left out (VariantShape::DR == 3),
// evaluated by the ray rule in a kernel of its own at arbitrary evaluation points (at the mesh's nodes the
// mesh walk takes them instead, bs_walk.cu).  Instantiated in bs_velocity.cu.
#pragma once

#include "bs_velocity_kernel.cuh"

namespace bs {
namespace {

// The near field as a pass of its own, after the far sweep of a variant with DR == 3 (which leaves the
// near pairs out of its sums).  One CTA per 32 consecutive points of the spatial order, one point per
// lane, with NW warps (kNearPassWarps; group g of 32 tiles to warp g mod NW); a batch gives every mesh its
// own CTAs (MeshDesc::near_warp_begin).  A warp tests its tiles with the far sweep's culling test against the
// points' bounding sphere; in each tile that can hold a near pair it classifies every (point, tet) pair with
// the far sweep's test (pair_is_near_*, the same decision bit for bit, so the near pass evaluates exactly the
// pairs the far sweep left out), and evaluates each near pair by the ray rule, the 32 lanes splitting its
// lines as in the fused drain (the float64 steps of the rare pairs that need them after the tet's pairs, where
// few registers are live).  The lane of the pair's point adds the result to its warp's total for that point
// (compensated in float32), in ascending tet order; the warps' totals are added in warp order (deterministic,
// independent of how the points are grouped) and written to near_out (float64, by spatial position), the ray
// hits to counts.  With a.near_split > 1 each group of 32 points has that many CTAs, CTA part s taking the
// tile groups s * NW + warp (mod NW * split); each part's totals go to its own slice of near_out and the
// reduction adds the slices in order.
template <typename T, int NW>
__global__ void __launch_bounds__(32 * NW, 16 / NW) near_pass_kernel(const VelocityArgs a)
{
    constexpr bool F32 = sizeof(T) == 4;
    __shared__ float spts[32 * 9];                   // the 32 points as float splits
    __shared__ float4 srec[NW][kNearF32Vec4];        // the near record of a warp's current tet
    __shared__ double stot[NW][32][3];               // the warps' totals
    __shared__ int shits[NW][32];
    extern __shared__ __align__(16) float4 sdir[];   // float32 direction table (a.smem_lines)
    if ((a.skip && *a.skip) || (a.near_skip && *a.near_skip)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (F32 && a.smem_lines)
        for (int l = threadIdx.x; l < a.L; l += blockDim.x) sdir[l] = a.lines.f32[l];
    // this CTA's group of 32 points over all meshes, and its part of the tiles (one mesh only)
    const int split = a.meshes ? 1 : max(a.near_split, 1);
    const int64_t wg = blockIdx.x / split;
    const int part = (int)(blockIdx.x % split);
    const MeshDesc *m = &a.m;
    if (a.meshes) {
        int lo = 0, hi = a.n_meshes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.meshes[mid].near_warp_begin <= wg) lo = mid;
            else hi = mid - 1;
        }
        m = &a.meshes[lo];
        if (a.mesh_near_skip && a.mesh_near_skip[lo] && *a.mesh_near_skip[lo]) return;  // the mesh's walk did it
    }
    const int64_t k = m->k;
    const int64_t w = wg - (a.meshes ? m->near_warp_begin : 0);
    if (w * 32 >= k || m->n_tets == 0) return;  // CTA-uniform
    const int64_t gi = w * 32 + lane;
    const int64_t gp = gi < k ? gi : k - 1;  // pad with a real point; its result is not written
    if (warp == 0) {
        const int64_t src = m->perm[gp];
#pragma unroll
        for (int j = 0; j < 3; ++j) split3(m->pts[3 * src + j], spts[9 * lane + 3 * j], spts[9 * lane + 3 * j + 1],
                                           spts[9 * lane + 3 * j + 2]);
    }
    __syncthreads();
    const float *xs = spts + 9 * lane;
    // bounding sphere of the 32 points (float, padded), as the far sweep's
    float4 sphere;
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
        const float ex = mxx - mnx, ey = mxy - mny, ez = mxz - mnz;
        sphere = make_float4(0.5f * (mnx + mxx), 0.5f * (mny + mxy), 0.5f * (mnz + mxz),
                             0.5f * sqrtf(ex * ex + ey * ey + ez * ez) * 1.001f + 1e-6f);
    }
    const float4 *lines = (F32 && a.smem_lines) ? sdir : a.lines.f32;
    const int tile = a.tile, rs = a.far_stride;
    const int64_t n_tiles = (m->n_tets + tile - 1) / tile;
    const V3<double> xd = mk(join3(xs[0], xs[1], xs[2]), join3(xs[3], xs[4], xs[5]), join3(xs[6], xs[7], xs[8]));
    float s32[3] = {0.f, 0.f, 0.f}, c32[3] = {0.f, 0.f, 0.f};  // float32: compensated total
    double s64[3] = {0.0, 0.0, 0.0};                            // float64: plain total
    int hits = 0;
    auto add = [&](float vx, float vy, float vz) {
        const float v[3] = {vx, vy, vz};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float y = v[q] - c32[q];
            const float s2 = s32[q] + y;
            c32[q] = (s2 - s32[q]) - y;
            s32[q] = s2;
        }
    };
#pragma unroll 1
    for (int64_t t0 = 32 * ((int64_t)part * NW + warp); t0 < n_tiles; t0 += 32 * (int64_t)NW * split) {
        const int64_t tl = t0 + lane;
        bool open = false;
        if (tl < n_tiles) open = a.all_ray || !tile_culled(sphere, m->tile_hdr[2 * tl], m->tile_hdr[2 * tl + 1].x,
                                                           a.far_ratio_f);
        unsigned tiles = __ballot_sync(0xffffffffu, open);
#pragma unroll 1
        while (tiles) {
            const int64_t t = t0 + __ffs(tiles) - 1;
            tiles &= tiles - 1u;
            const float4 o = m->tile_hdr[2 * t];
            const int cnt = (int)min((int64_t)tile, m->n_tets - t * tile);
            const float xp = xs[0] - o.x, yp = xs[3] - o.y, zp = xs[6] - o.z;  // tile frame (float32)
#pragma unroll 1
            for (int j0 = 0; j0 < cnt; j0 += 32) {
                // lane jj holds the decision data of tet j0 + jj of the tile
                const int64_t tj = t * tile + j0 + lane;
                float4 c32v = make_float4(0.f, 0.f, 0.f, 0.f);
                double c64v[4] = {0.0, 0.0, 0.0, 0.0};
                if (j0 + lane < cnt) {
                    if constexpr (F32) {
                        c32v = *reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(m->far) + tj * rs);
                    } else {
                        const double *r = reinterpret_cast<const double *>(m->far) + tj * rs;
#pragma unroll
                        for (int q = 0; q < 4; ++q) c64v[q] = r[q];
                    }
                }
                const int nj = min(32, cnt - j0);
#pragma unroll 1
                for (int jj = 0; jj < nj; ++jj) {
                    bool nearp;
                    if constexpr (F32) {
                        float4 c;
                        c.x = __shfl_sync(0xffffffffu, c32v.x, jj);
                        c.y = __shfl_sync(0xffffffffu, c32v.y, jj);
                        c.z = __shfl_sync(0xffffffffu, c32v.z, jj);
                        c.w = __shfl_sync(0xffffffffu, c32v.w, jj);
                        nearp = pair_is_near_f32(xp, yp, zp, c, a.far_ratio2_f);
                    } else {
                        double c[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) c[q] = __shfl_sync(0xffffffffu, c64v[q], jj);
                        nearp = pair_is_near_f64(xd.x, xd.y, xd.z, c, a.far_ratio2);
                    }
                    unsigned owners = __ballot_sync(0xffffffffu, nearp && gi < k);
                    if (!owners) continue;
                    const int64_t tet = t * tile + j0 + jj;
                    if constexpr (F32) {
                        __syncwarp();
                        if (lane < kNearF32Vec4) srec[warp][lane] = m->near32[tet * kNearF32Vec4 + lane];
                        __syncwarp();
                        unsigned redo = 0u;  // owners whose pair needs the float64 steps
#pragma unroll 1
                        for (unsigned ow = owners; ow; ow &= ow - 1u) {
                            const int owner = __ffs(ow) - 1;
                            bool rd = false, whole = false;
                            int vk = -1;
                            const NearOut32 r = near_pair_f32_body<1, true>(spts + 9 * owner, srec[warp],
                                                                            m->near64 + tet * kNearF64, lines,
                                                                            a.lines.f64, a.L, lane, &rd, &vk, &whole);
                            if (lane == owner) {
                                add(r.vx, r.vy, r.vz);
                                hits += r.hits;
                            }
                            if (rd) redo |= 1u << owner;
                        }
#pragma unroll 1
                        for (; redo; redo &= redo - 1u) {  // rare
                            const int owner = __ffs(redo) - 1;
                            const float *xo = spts + 9 * owner;
                            const V3<double> x = mk(join3(xo[0], xo[1], xo[2]), join3(xo[3], xo[4], xo[5]),
                                                    join3(xo[6], xo[7], xo[8]));
                            // vertex index and whole-pair decision again (the same float32 tests)
                            const float *vh = reinterpret_cast<const float *>(srec[warp] + nf32::VH);
                            const float *vm = reinterpret_cast<const float *>(srec[warp] + nf32::VM);
                            int vk = -1;
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                if (vk < 0 && vh[3 * i] == xo[0] && vm[3 * i] == xo[1] && vh[3 * i + 1] == xo[3] &&
                                    vm[3 * i + 1] == xo[4] && vh[3 * i + 2] == xo[6] && vm[3 * i + 2] == xo[7])
                                    vk = i;
                            bool whole = false;
                            if (vk < 0) {
                                const float4 q0 = srec[warp][nf32::G1], q1 = srec[warp][nf32::G2],
                                             q2 = srec[warp][nf32::G3];
                                const V3<float> d0 = mk((xo[0] - vh[0]) + (xo[1] - vm[0]), (xo[3] - vh[1]) + (xo[4] - vm[1]),
                                                        (xo[6] - vh[2]) + (xo[7] - vm[2]));
                                float av[4];
                                av[1] = q0.x * d0.x + q0.y * d0.y + q0.z * d0.z;
                                av[2] = q1.x * d0.x + q1.y * d0.y + q1.z * d0.z;
                                av[3] = q2.x * d0.x + q2.y * d0.y + q2.z * d0.z;
                                av[0] = 1.0f - av[1] - av[2] - av[3];
                                const float amin = fminf(fminf(av[0], av[1]), fminf(av[2], av[3]));
                                const float aabs = fminf(fminf(fabsf(av[0]), fabsf(av[1])), fminf(fabsf(av[2]), fabsf(av[3])));
                                whole = amin > -kDegenA && aabs < kDegenA;
                            }
                            V3<double> acc = mk(0.0, 0.0, 0.0);
                            int h2 = 0;
                            line_fallback_f64_inl(x, xo, srec[warp], m->near64 + tet * kNearF64, lines, a.lines.f64,
                                                  a.L, lane, vk, whole, acc, h2);
                            const double vx = warp_sum(acc.x), vy = warp_sum(acc.y), vz = warp_sum(acc.z);
                            h2 = warp_sum(h2);
                            if (lane == owner) {
                                add((float)vx, (float)vy, (float)vz);
                                hits += h2;
                            }
                        }
                    } else {
#pragma unroll 1
                        for (; owners; owners &= owners - 1u) {
                            const int owner = __ffs(owners) - 1;
                            const V3<double> xo = mk(__shfl_sync(0xffffffffu, xd.x, owner),
                                                     __shfl_sync(0xffffffffu, xd.y, owner),
                                                     __shfl_sync(0xffffffffu, xd.z, owner));
                            const NearOut r = near_pair_f64(xo, m->near64 + tet * kNearF64, a.lines.f64, a.L, lane);
                            if (lane == owner) {
                                s64[0] += r.vx;
                                s64[1] += r.vy;
                                s64[2] += r.vz;
                                hits += r.hits;
                            }
                        }
                    }
                }
            }
        }
    }
    // the four warps' totals, added in warp order
#pragma unroll
    for (int q = 0; q < 3; ++q) stot[warp][lane][q] = F32 ? (double)s32[q] - (double)c32[q] : s64[q];
    shits[warp][lane] = hits;
    __syncthreads();
    if (warp != 0 || gi >= k) return;
    double tot[3] = {0.0, 0.0, 0.0};
    int th = 0;
#pragma unroll
    for (int v = 0; v < NW; ++v) {
#pragma unroll
        for (int q = 0; q < 3; ++q) tot[q] += stot[v][lane][q];
        th += shits[v][lane];
    }
    double *dst = a.near_out + part * a.near_split_stride + 3 * ((a.meshes ? m->point_begin : 0) + gi);
#pragma unroll
    for (int q = 0; q < 3; ++q) dst[q] = tot[q];
    if (a.counts) {
        if (split == 1) a.counts[3 * m->perm[gi] + 2] += th;
        else atomicAdd(&a.counts[3 * m->perm[gi] + 2], th);  // integer sum: order-independent
    }
}

}  // namespace
}  // namespace bs
