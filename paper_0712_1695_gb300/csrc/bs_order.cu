// bs_order.cu -- spatial ordering of the evaluation points.
//
// The velocity kernel gives each warp a run of consecutive points and tests
// whole tet tiles against the warp's bounding sphere (a tile that is far
// from every point of the warp needs no per-pair near/far test).  That only
// pays when a warp's points are close together, so the points are visited
// in Morton (Z-curve) order of a cell grid over their bounding box: a
// counting sort by cell.  The order inside a cell comes from atomics and is
// not deterministic, but no result depends on it: each point's sum runs
// over the tets in the same order whatever block the point lands in.
#include <math.h>

#include <algorithm>

#include "bs_internal.cuh"

namespace bs {
namespace {

__device__ inline unsigned spread3(unsigned v)  // 10 bits -> every third bit of 30
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// float -> int mapping that preserves order (for atomicMin/atomicMax on floats)
__device__ inline int f2ord(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ inline float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void bbox_kernel(const double *__restrict__ pts, int64_t k, int *box)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < 3; ++j) {
            const float v = (float)pts[3 * i + j];
            lo[j] = fminf(lo[j], v);
            hi[j] = fmaxf(hi[j], v);
        }
    for (int j = 0; j < 3; ++j)
        for (int o = 16; o > 0; o >>= 1) {
            lo[j] = fminf(lo[j], __shfl_xor_sync(0xffffffffu, lo[j], o));
            hi[j] = fmaxf(hi[j], __shfl_xor_sync(0xffffffffu, hi[j], o));
        }
    if ((threadIdx.x & 31) == 0)
        for (int j = 0; j < 3; ++j) {
            atomicMin(&box[j], f2ord(lo[j]));
            atomicMax(&box[3 + j], f2ord(hi[j]));
        }
}

__global__ void key_count_kernel(const double *__restrict__ pts, int64_t k, const int *__restrict__ box, int bits,
                                 unsigned *__restrict__ keys, int *__restrict__ count)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= k) return;
    const int G = 1 << bits;
    unsigned c[3];
    for (int j = 0; j < 3; ++j) {
        const float lo = ord2f(box[j]), hi = ord2f(box[3 + j]);
        const float span = hi - lo;
        const float u = span > 0.f ? ((float)pts[3 * i + j] - lo) / span : 0.f;
        int ci = (int)(u * G);
        ci = ci < 0 ? 0 : (ci >= G ? G - 1 : ci);
        c[j] = (unsigned)ci;
    }
    const unsigned key = spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
    keys[i] = key;
    atomicAdd(&count[key], 1);
}

// exclusive scan of n counts by one block (n up to a few million: each thread scans a contiguous run)
__global__ void scan_kernel(int *__restrict__ count, int n)
{
    __shared__ int part[1024];
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per, e = min(b + per, n);
    int s = 0;
    for (int i = b; i < e; ++i) s += count[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int v = part[t];
            part[t] = run;
            run += v;
        }
    }
    __syncthreads();
    int run = part[threadIdx.x];
    for (int i = b; i < e; ++i) {
        const int v = count[i];
        count[i] = run;
        run += v;
    }
}

__global__ void scatter_kernel(const unsigned *__restrict__ keys, int64_t k, int *__restrict__ offset,
                               int *__restrict__ perm)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= k) return;
    const int pos = atomicAdd(&offset[keys[i]], 1);
    perm[pos] = (int)i;
}

__global__ void init_box_kernel(int *box)
{
    if (threadIdx.x < 3) {
        box[threadIdx.x] = f2ord(INFINITY);
        box[3 + threadIdx.x] = f2ord(-INFINITY);
    }
}

}  // namespace

// cells ~ k/8 (about eight points per cell: a warp's 32-64 points still span only a few cells)
int order_grid_bits(int64_t k)
{
    int bits = 1;
    while (bits < 7 && ((int64_t)1 << (3 * bits)) < (k + 7) / 8) ++bits;
    return bits;
}

cudaError_t spatial_order(const double *pts, int64_t k, int bits, int *box, unsigned *keys, int *count, int *perm,
                          cudaStream_t st)
{
    const int cells = 1 << (3 * bits);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * cells, st);
    if (e != cudaSuccess) return e;
    init_box_kernel<<<1, 32, 0, st>>>(box);
    const int tb = 256;
    const int nb = (int)std::min<int64_t>((k + tb - 1) / tb, 1024);
    bbox_kernel<<<nb, tb, 0, st>>>(pts, k, box);
    key_count_kernel<<<(unsigned)((k + tb - 1) / tb), tb, 0, st>>>(pts, k, box, bits, keys, count);
    scan_kernel<<<1, 1024, 0, st>>>(count, cells);
    scatter_kernel<<<(unsigned)((k + tb - 1) / tb), tb, 0, st>>>(keys, k, count, perm);
    return cudaGetLastError();
}

}  // namespace bs
