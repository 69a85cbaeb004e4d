// bs_noalloc.cu -- bs_velocity_noalloc: velocity evaluation that allocates no
// device memory.
//
// Who needs it: callers that must not let a library allocate GPU memory, for
// example an application that hands all device memory to its own pool or
// arena and accounts for every byte, or a simulation loop that cannot afford
// the device synchronisation or the out-of-memory failure a driver
// allocation may bring in the middle of a run.  bs_create / bs_velocity
// allocate the mesh tables, the direction table and the partial sums
// themselves; this entry point instead works from the caller's device arrays
// and keeps every table and partial sum in one fixed array of device memory
// that belongs to the library (g_scratch below).  That array exists on every
// GPU that loads the library, for the life of the process, whether or not
// this entry point is used.
//
// Limits (anything larger is rejected with BS_ERR_ARG): kMaxTets tets,
// kMaxPoints evaluation points, kMaxLines = n_theta * n_phi directions, tet
// rules with 1 or 4 points.
//
// Errors found on the device: the mesh is not validated on the host (that
// would need a synchronisation).  A node index out of range, a degenerate tet
// (|volume| <= 1e-14 h^3) or a bulk-copy wait that gave up raises a flag in
// the scratch array, and the call's last kernel then overwrites every
// velocity with NaN and every count with -1.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "bs_internal.cuh"

namespace {

using namespace bs;

constexpr int64_t kMaxTets = 8192;
constexpr int64_t kMaxPoints = 4096;
constexpr int64_t kMaxLines = 4096;
constexpr int kMaxQ = 4;
constexpr int kMaxChunks = 32;
constexpr int kMaxCellBits = 4;  // spatial order grid of 16^3 cells (enough for kMaxPoints)
constexpr int kMaxTile = 32;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets of the pieces inside the scratch array
constexpr size_t kNear32 = 0;
constexpr size_t kNear64 = kNear32 + align256(kMaxTets * kNearF32Vec4 * sizeof(float4));
constexpr size_t kRho2 = kNear64 + align256(kMaxTets * kNearF64 * sizeof(double));
constexpr size_t kFar32 = kRho2 + align256(kMaxTets * sizeof(double));
constexpr size_t kFar64 = kFar32 + align256(kMaxTets * far_stride<float>(kMaxQ) * sizeof(float));
constexpr size_t kHdr = kFar64 + align256(kMaxTets * far_stride<double>(kMaxQ) * sizeof(double));
constexpr size_t kBary = kHdr + align256((kMaxTets / 8 + 1) * 2 * sizeof(float4));  // tiles of >= 8 tets
constexpr size_t kWq = kBary + align256(4 * kMaxQ * sizeof(double));
constexpr size_t kLines32 = kWq + align256(kMaxQ * sizeof(double));
constexpr size_t kLines64 = kLines32 + align256(kMaxLines * sizeof(float4));
constexpr size_t kPerm = kLines64 + align256(kMaxLines * sizeof(dbl4));
constexpr size_t kKeys = kPerm + align256(kMaxPoints * sizeof(int));
constexpr size_t kCells = kKeys + align256(kMaxPoints * sizeof(unsigned));
constexpr size_t kBox = kCells + align256(sizeof(int) << (3 * kMaxCellBits));
constexpr size_t kPartial = kBox + align256(8 * sizeof(int));
constexpr size_t kFlag = kPartial + align256((size_t)kMaxChunks * kMaxPoints * 3 * sizeof(double));
constexpr size_t kFirstBad = kFlag + align256(sizeof(int));
constexpr size_t kCounter = kFirstBad + align256(sizeof(unsigned long long));
constexpr size_t kScratchBytes = kCounter + align256(sizeof(unsigned long long));

// The library's fixed scratch memory (about 11 MB).  Host code must not take
// its address directly: the name is a host-side stand-in, so the device
// address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_addr[64] = {};  // device address of g_scratch, per device ordinal

// Runs after the reduction: if any kernel of this call raised the error flag (a node index out of range,
// a degenerate tet, a bulk-copy wait that gave up), the whole output becomes NaN and the counts -1.  The
// caller learns of the error from its own results without a synchronisation or a status call.
__global__ void poison_kernel(const int *flag, double *out, int32_t *counts, int64_t k)
{
    if (*flag == 0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * k; i += (int64_t)gridDim.x * blockDim.x) {
        out[i] = __longlong_as_double(0x7ff8000000000000LL);  // quiet NaN
        if (counts) counts[i] = -1;
    }
}

}  // namespace

// Errors are reported through bs_last_error() like every other call.
void bs_set_last_error(const char *msg);

extern "C" int bs_velocity_noalloc(const double *nodes_dev, int64_t n_nodes, const int32_t *tets_dev, int64_t n_tets,
                        const double *omega_dev, const double *eval_pts_dev, int64_t k, const bs_params *p,
                        double *out_dev, void *stream)
{
    auto fail = [](int code, const char *msg) {
        bs_set_last_error(msg);
        return code;
    };
    if (!p) return fail(BS_ERR_ARG, "bs_velocity_noalloc: params is NULL");
    if (!nodes_dev || !omega_dev || !eval_pts_dev || !out_dev || (n_tets > 0 && !tets_dev))
        return fail(BS_ERR_ARG, "bs_velocity_noalloc: NULL array");
    if (n_nodes < 1 || n_tets < 0 || k < 0) return fail(BS_ERR_ARG, "bs_velocity_noalloc: bad sizes");
    if (n_nodes > INT32_MAX) return fail(BS_ERR_ARG, "bs_velocity_noalloc: n_nodes exceeds the int32 index range");
    if (n_tets > kMaxTets) return fail(BS_ERR_ARG, "bs_velocity_noalloc: more than 8192 tets (fixed scratch limit)");
    if (k > kMaxPoints)
        return fail(BS_ERR_ARG, "bs_velocity_noalloc: more than 4096 evaluation points (fixed scratch limit)");
    const double fr = p->far_ratio;
    if (isnan(fr) || (!isinf(fr) && fr < 2.0) || (isinf(fr) && fr < 0))
        return fail(BS_ERR_ARG, "bs_velocity_noalloc: far_ratio must be >= 2 or +INFINITY");
    if (p->n_theta < 1 || p->n_theta > 256 || p->n_phi < 1 || p->n_phi > 256)
        return fail(BS_ERR_ARG, "bs_velocity_noalloc: n_theta and n_phi must be in 1..256");
    if ((int64_t)p->n_theta * p->n_phi > kMaxLines)
        return fail(BS_ERR_ARG, "bs_velocity_noalloc: n_theta * n_phi above 4096 (fixed scratch limit)");
    if (p->precision != BS_FP32 && p->precision != BS_FP64)
        return fail(BS_ERR_ARG, "bs_velocity_noalloc: precision must be BS_FP64 or BS_FP32");
    if (p->near_rule != BS_NEAR_RAY && p->near_rule != BS_NEAR_EXACT)
        return fail(BS_ERR_ARG, "bs_velocity_noalloc: near_rule must be BS_NEAR_RAY or BS_NEAR_EXACT");
    if (p->tet_gauss_order != 1 && p->tet_gauss_order != 4)
        return fail(BS_ERR_ORDER, "bs_velocity_noalloc: tet_gauss_order must be 1 or 4 (fixed scratch limit)");
    if (k == 0) return BS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    auto cuda_fail = [&](cudaError_t e, const char *where) {
        static thread_local std::string m;
        m = std::string("bs_velocity_noalloc: ") + where + ": " + cudaGetErrorString(e);
        bs_set_last_error(m.c_str());
        return BS_ERR_CUDA;
    };

    // one-time set-up per device: the device address of the scratch array
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(BS_ERR_ARG, "bs_velocity_noalloc: device ordinal above 63");
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
            g_addr[dev] = static_cast<unsigned char *>(ptr);
        }
        base = g_addr[dev];
    }
    int n_sm = 0;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "cudaDeviceGetAttribute");

    if (n_tets == 0) {
        if ((e = cudaMemsetAsync(out_dev, 0, sizeof(double) * 3 * k, st)) != cudaSuccess)
            return cuda_fail(e, "cudaMemsetAsync");
        if (p->counts && (e = cudaMemsetAsync(p->counts, 0, sizeof(int32_t) * 3 * k, st)) != cudaSuccess)
            return cuda_fail(e, "cudaMemsetAsync");
        return BS_OK;
    }

    float4 *near32 = reinterpret_cast<float4 *>(base + kNear32);
    double *near64 = reinterpret_cast<double *>(base + kNear64);
    double *rho2 = reinterpret_cast<double *>(base + kRho2);
    float *far32 = reinterpret_cast<float *>(base + kFar32);
    double *far64 = reinterpret_cast<double *>(base + kFar64);
    float4 *hdr = reinterpret_cast<float4 *>(base + kHdr);
    int *flag = reinterpret_cast<int *>(base + kFlag);
    unsigned long long *first_bad = reinterpret_cast<unsigned long long *>(base + kFirstBad);
    TetRule rule;
    rule.order = p->tet_gauss_order;
    rule.bary = reinterpret_cast<double *>(base + kBary);
    rule.w = reinterpret_cast<double *>(base + kWq);
    LineTables lines;
    lines.n_phi = p->n_phi;
    lines.n_theta = p->n_theta;
    lines.f32 = reinterpret_cast<float4 *>(base + kLines32);
    lines.f64 = reinterpret_cast<dbl4 *>(base + kLines64);

    const int Q = p->tet_gauss_order;
    // meshes within the fixed limits are small: the one-point-per-thread variant where there is one, and a
    // variant whose far records and tile headers fit the scratch layout
    const int variant = noalloc_variant(p->precision, Q, p->near_rule);
    const LaunchShape shape = shape_for(p->precision, Q, variant, p->near_rule);
    if (variant < 0 || shape.tile > kMaxTile || shape.tile < 8 || shape.layout != kFarQuadPairs)
        return fail(BS_ERR_ARG, "bs_velocity_noalloc: no kernel variant fits the scratch layout");

    // the per-call state that must start from zero / "none"
    if ((e = cudaMemsetAsync(flag, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if ((e = cudaMemsetAsync(first_bad, 0xff, sizeof(unsigned long long), st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync");

    // tables (the same kernels bs_create / bs_velocity use, writing into the scratch array)
    if ((e = build_near_records(nodes_dev, n_nodes, tets_dev, n_tets, omega_dev, near32, near64, rho2, flag,
                                first_bad, st)) != cudaSuccess)
        return cuda_fail(e, "near records");
    if ((e = build_tet_rule(Q, rule.bary, rule.w, st)) != cudaSuccess) return cuda_fail(e, "tet rule");
    if ((e = build_far_records(near64, rho2, n_tets, rule, shape.tile, kFarQuadPairs, hdr, far32, far64, st)) !=
        cudaSuccess)
        return cuda_fail(e, "far records");
    if ((e = build_lines(p->n_phi, p->n_theta, lines.f32, lines.f64, st)) != cudaSuccess)
        return cuda_fail(e, "direction table");

    // decomposition, as in bs_velocity but with at most kMaxChunks chunks
    const int occ = std::max(1, velocity_ctas_per_sm(p->precision, Q, variant, p->near_rule));
    const int64_t BP = (int64_t)shape.threads * shape.points_per_thread;
    const int64_t n_blocks = (k + BP - 1) / BP;
    const int64_t n_tiles = (n_tets + shape.tile - 1) / shape.tile;
    const int64_t target = 16LL * n_sm * occ;
    int64_t n_chunks = std::min<int64_t>(std::max<int64_t>((target + n_blocks - 1) / n_blocks, 1), n_tiles);
    n_chunks = std::min<int64_t>(n_chunks, kMaxChunks);
    // at least kMinTilesPerItem tiles per item: shorter items are dominated by their set-up
    const int64_t per = std::min<int64_t>(std::max<int64_t>((n_tiles + n_chunks - 1) / n_chunks, kMinTilesPerItem),
                                          n_tiles);
    n_chunks = (n_tiles + per - 1) / per;

    const int bits = std::min(order_grid_bits(k), kMaxCellBits);
    int *perm = reinterpret_cast<int *>(base + kPerm);
    if ((e = spatial_order(eval_pts_dev, k, bits, reinterpret_cast<int *>(base + kBox),
                           reinterpret_cast<unsigned *>(base + kKeys), reinterpret_cast<int *>(base + kCells), perm,
                           st)) != cudaSuccess)
        return cuda_fail(e, "spatial order");

    VelocityArgs a;
    a.m.n_tets = n_tets;
    a.m.far = p->precision == BS_FP32 ? (const void *)far32 : (const void *)far64;
    a.m.near32 = near32;
    a.m.near64 = near64;
    a.m.tile_hdr = hdr;
    a.m.pts = eval_pts_dev;
    a.m.perm = perm;
    a.m.k = k;
    a.Q = Q;
    set_far_ratio(a, fr);
    a.lines = lines;
    a.L = p->n_phi * p->n_theta;
    a.smem_lines = a.L <= kSmemLinesMax ? 1 : 0;
    a.counts = p->counts;
    a.m.out = out_dev;
    a.flag = flag;
    a.work_counter = reinterpret_cast<unsigned long long *>(base + kCounter);
    a.m.n_chunks = (int)n_chunks;
    a.m.tiles_per_chunk = (int)per;
    a.m.partial = reinterpret_cast<double *>(base + kPartial);
    a.variant = variant;
    a.near_rule = p->near_rule;
    a.n_items = n_blocks * n_chunks;
    int grid = 0;
    if ((e = launch_velocity(p->precision, a, n_sm, st, &grid)) != cudaSuccess) return cuda_fail(e, "velocity");
    if ((e = launch_reduce(a, st)) != cudaSuccess) return cuda_fail(e, "reduce");
    poison_kernel<<<(unsigned)std::min<int64_t>((3 * k + 255) / 256, 1024), 256, 0, st>>>(flag, out_dev, p->counts, k);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "poison");
    return BS_OK;
}

extern "C" int bs_noalloc_status(void *stream, int64_t *first_bad_tet)
{
    if (first_bad_tet) *first_bad_tet = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        bs_set_last_error(cudaGetErrorString(e));
        return BS_ERR_CUDA;
    }
    if (dev < 0 || dev >= 64) {
        bs_set_last_error("bs_noalloc_status: device ordinal above 63");
        return BS_ERR_ARG;
    }
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        base = g_addr[dev];
    }
    if (!base) return BS_OK;  // no bs_velocity_noalloc call on this device yet: nothing to report
    // the flag word and the lowest bad tet, read in stream order after the calls queued before this one
    cudaStream_t st = (cudaStream_t)stream;
    int flag = 0;
    unsigned long long bad = ~0ULL;
    if ((e = cudaMemcpyAsync(&flag, base + kFlag, sizeof flag, cudaMemcpyDeviceToHost, st)) == cudaSuccess &&
        (e = cudaMemcpyAsync(&bad, base + kFirstBad, sizeof bad, cudaMemcpyDeviceToHost, st)) == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        static thread_local std::string m;
        m = std::string("bs_noalloc_status: ") + cudaGetErrorString(e);
        bs_set_last_error(m.c_str());
        return BS_ERR_CUDA;
    }
    if (flag & (kFlagMeshIndex | kFlagMeshVolume)) {
        if (first_bad_tet && bad != ~0ULL) *first_bad_tet = (int64_t)bad;
        bs_set_last_error((flag & kFlagMeshIndex) ? "bs_velocity_noalloc: node index out of range (or degenerate tet)"
                                                  : "bs_velocity_noalloc: degenerate tet");
        return BS_ERR_MESH;
    }
    if (flag & kFlagTimeout) {
        bs_set_last_error("bs_velocity_noalloc: a bounded device wait gave up");
        return BS_ERR_TIMEOUT;
    }
    return BS_OK;
}
