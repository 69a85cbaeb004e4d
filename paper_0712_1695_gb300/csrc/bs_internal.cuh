// bs_internal.cuh -- device data layouts and helpers shared by the libbs
// translation units (tables, per-tet precompute, velocity kernels, C ABI).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bs.h"

namespace bs {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Per-tet records.
//
// Far record (one per tet, rebuilt when the far rule changes): everything the
// far rule and the near/far test need, streamed through shared memory, with
// w'_q = -(w_q |V| / 4pi) omega(x_q) (sign and 1/4pi of Eq. 1 folded in).
//   double: [c (3), rho^2] then per quadrature point [x_q (3), w'_q (3)]  (4 + 6Q)
//   float : tile frame (coordinates relative to the tile origin o), in one of two layouts:
//           quadrature-pair layout: [c - o (3), rho^2] then the quadrature points in pairs (a, b),
//           five float4 per pair, every value stored as the pair (value_a, value_b) so that one
//           packed f32x2 instruction serves both points:
//           [-2x'.x, -2x'.y] [-2x'.z, |x'|^2] [w'.x, w'.y] [w'.z, B.x] [B.y, B.z]
//           (B = x_q' x w'_q; an odd Q is padded with a point of zero weight)  (4 + 20 ceil(Q/2));
//           point-pair layout: the same five float4 per quadrature point with every value
//           stored twice, (value, value), so that one packed instruction serves two evaluation
//           points  (4 + 20 Q)
// Tile header (per TILE consecutive tets): float4 [o (3), rc], float4 [rho_max, 0, 0, 0].
//
// Near record (one per tet, independent of the parameters): what the ray rule
// needs.  Barycentric coordinates lambda_i(y) = g_i . (y - v0) + delta_i0
// with g_0 = -(g_1 + g_2 + g_3) (the face planes of the tet).
//   float  : 15 x float4  [g1 h] [g2 Rb^2] [g3 -] [w0 -] [w1 -] [w2 -] [w3 -]
//            [c hi (3) -] [c mid (3) -] [vertex hi: 12 floats] [vertex mid: 12 floats]
//            (coordinates as float splits x = hi + mid + lo, see split3: the float path
//            takes differences and vertex tests without float64 arithmetic)
//   double : 40 doubles  v0..v3 (12) g1 g2 g3 (9) w0..w3 (12) c (3) h Rb^2 (2) pad (2)
//   h = longest edge, c = centroid, Rb = largest vertex distance from c.
// ---------------------------------------------------------------------------
constexpr int kFarQuadPairs = 0;   // float32 far-record layouts (see above)
constexpr int kFarPointPairs = 1;
template <typename T>
__host__ __device__ constexpr int far_stride(int Q, int layout = kFarQuadPairs)
{
    return sizeof(T) == 4 ? (layout == kFarPointPairs ? 4 + 20 * Q : 4 + 20 * ((Q + 1) / 2)) : (4 + 10 * Q);
}
constexpr int kNearF32Vec4 = 15;  // float4 per near record
namespace nf32 {
constexpr int G1 = 0, G2 = 1, G3 = 2, W = 3, CH = 7, CM = 8, VH = 9, VM = 12;  // float4 index
}

// x = hi + mid + lo exactly (three floats hold the 53 bits of a normal double):
// hi = fl(x), mid = fl(x - hi), lo = fl(x - hi - mid); each difference is exact.
__host__ __device__ inline void split3(double x, float &hi, float &mid, float &lo)
{
    hi = (float)x;
    const double r = x - (double)hi;
    mid = (float)r;
    lo = (float)(r - (double)mid);
}
__host__ __device__ inline double join3(float hi, float mid, float lo)
{
    return ((double)hi + (double)mid) + (double)lo;
}
constexpr int kNearF64 = 40;     // doubles per near record
namespace nf64 {
constexpr int V = 0, G = 12, W = 21, C = 33, H = 36, RB2 = 37;
}

// Four doubles on a 32-byte boundary (one line of the direction table).
struct __align__(32) dbl4 {
    double x, y, z, w;
};

// Line table of Eq. 3: per line (s_x, s_y, s_z, k) in float4 and dbl4.
struct LineTables {
    int n_phi = 0, n_theta = 0;
    float4 *f32 = nullptr;
    dbl4 *f64 = nullptr;
};

struct TetRule {
    int order = 0;
    double *bary = nullptr;  // device [order][4]
    double *w = nullptr;     // device [order]
};

// Error flag values written by kernels (device int in the handle).
constexpr int kFlagMeshIndex = 1;
constexpr int kFlagMeshVolume = 2;
constexpr int kFlagTimeout = 4;
constexpr int kFlagWalk = 8;     // a mesh walk hit its step limit or a tet with no face ahead
constexpr int kFlagNoWalk = 16;  // a derivative along directions was asked of a mesh the walk cannot serve
constexpr int kFlagWalkStuck = 32;  // a mesh walk reached a tet with no face ahead of the line

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).
// ---------------------------------------------------------------------------
cudaError_t build_lines(int n_phi, int n_theta, float4 *f32, dbl4 *f64, cudaStream_t st);
cudaError_t build_tet_rule(int order, double *bary, double *w, cudaStream_t st);

// near records + per-tet validity; error flag gets kFlagMesh* and first_bad the lowest bad tet
cudaError_t build_near_records(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                               const double *omega, float4 *near32, double *near64, double *rho2,
                               int *flag, unsigned long long *first_bad, cudaStream_t st);
// tile headers and far records for a tet rule, tile size and float32 layout (needs near64 and rho2)
cudaError_t build_far_records(const double *near64, const double *rho2, int64_t n_tets, const TetRule &rule,
                              int tile, int layout32, float4 *hdr, float *far32, double *far64, cudaStream_t st);
// spatial order of the evaluation points (Morton counting sort on a 2^bits grid)
int order_grid_bits(int64_t k);
cudaError_t spatial_order(const double *pts, int64_t k, int bits, int *box, unsigned *keys, int *count, int *perm,
                          cudaStream_t st);

// One mesh of a launch: its tables, its evaluation points and where the
// per-chunk partial sums go.  A batch launch reads an array of these.
struct MeshDesc {
    const void *far = nullptr;  // far records (float or double)
    const float4 *near32 = nullptr;
    const double *near64 = nullptr;
    const float4 *tile_hdr = nullptr;  // [n_tiles][2] origin + centroid radius, largest circumradius
    const double *pts = nullptr;       // [k][3]
    const int *perm = nullptr;         // [k] visiting order (spatially sorted)
    double *partial = nullptr;         // [n_chunks][k][3]
    double *out = nullptr;             // [k][3]
    int64_t k = 0, n_tets = 0;
    int n_chunks = 1, tiles_per_chunk = 1;
    int64_t item_begin = 0;   // batch: first work item of this mesh
    int64_t point_begin = 0;  // batch: first point of this mesh in the batched reduction
    int64_t near_warp_begin = 0;  // batch: first warp of this mesh in the near pass
};

struct VelocityArgs {
    MeshDesc m;                        // single-mesh launch
    const MeshDesc *meshes = nullptr;  // batch launch: device array [n_meshes] (m unused)
    int n_meshes = 0;
    int64_t n_items = 0;   // work items (point block x tet chunk) over all meshes
    int64_t n_points = 0;  // batch: points over all meshes
    // rule
    int Q = 4;
    double far_ratio2 = 4.0;  // +inf for all-ray
    float far_ratio2_f = 4.0f, far_ratio_f = 2.0f;  // the same in float, and the far ratio (+inf for all-ray)
    int all_ray = 0;
    LineTables lines;
    int L = 0;
    int smem_lines = 0;  // the float32 direction table is copied to shared memory (set for small L)
    // outputs
    int32_t *counts = nullptr;  // [k][3] or null (single mesh only; zeroed before)
    int *flag = nullptr;
    unsigned long long *work_counter = nullptr;  // device item counter, zeroed by launch_velocity
    int variant = 0;  // kernel variant (points per thread / registers) for this precision and rule
    const int *skip = nullptr;  // device flag: when set, the all-ray and reduce kernels return at once
    int near_rule = 0;          // BS_NEAR_RAY or BS_NEAR_EXACT
    // bounded waits: polls of a bulk-copy wait before the kernel gives up (raises kFlagTimeout and
    // returns); withhold_copies = 1 arms the copy barriers without issuing the copies (a test of the
    // give-up path: nothing can land after the kernel returned)
    long long wait_polls = 0;
    int withhold_copies = 0;
    // the near pass (variants that leave the near pairs to it): float64 near totals by spatial position
    // ([n_points][3]; batch: over all meshes), the far records' tile and stride, and its number of warps
    double *near_out = nullptr;
    int tile = 0, far_stride = 0;
    int64_t n_near_warps = 0;  // groups of 32 points (one CTA of the near pass each)
    const int *near_skip = nullptr;  // device flag: when set, the near pass returns at once
    // one mesh (not a batch), no mesh walk: the tiles split into near_split interleaved parts, one CTA per
    // (group of 32 points, part), part s writing its totals to near_out + s * near_split_stride; the
    // reduction adds the parts in order
    int near_split = 1;
    int64_t near_split_stride = 0;
    // batch: per mesh, a device flag set when the mesh walk took that mesh's near field (or null)
    const int *const *mesh_near_skip = nullptr;
};

// the near pass: warps per CTA (one group of 32 points; one warp scanning every tile beat four warps
// sharing them, whose barrier waited on the one holding the group's near tiles), and the CTAs per SM a
// launch on few points aims for by splitting the tiles among several CTAs per group
constexpr int kNearPassWarps = 1;
constexpr int kNearPassBlocksPerSm = 32;
// side streams a batch's per-mesh near walks are spread over (graph branches that run concurrently)
constexpr int kBatchWalkStreams = 8;
static_assert(kBatchWalkStreams <= 32, "the forked side streams are a 32-bit mask");

// far ratio of a launch: its square (+inf for the all-ray rule) in double and float, the ratio in float
inline void set_far_ratio(VelocityArgs &a, double far_ratio)
{
    const bool inf = far_ratio > 1e300;
    a.far_ratio2 = inf ? (double)INFINITY : far_ratio * far_ratio;
    a.far_ratio2_f = (float)a.far_ratio2;
    a.far_ratio_f = inf ? INFINITY : (float)sqrt(a.far_ratio2);
    a.all_ray = inf ? 1 : 0;
}

constexpr int64_t kMinTilesPerItem = 2;  // work items shorter than this are dominated by their set-up
constexpr int kSmemLinesMax = 256;       // direction tables up to this many lines live in shared memory

struct LaunchShape {
    int points_per_thread = 2;  // P
    int threads = 128;
    int tile = 64;    // tets per shared-memory tile
    int layout = 0;   // float32 far-record layout (kFarQuadPairs / kFarPointPairs)
    int drain = 1;    // VariantShape::DR (3: the near pass evaluates the near pairs)
};

// Kernel variants of the velocity kernel, per (precision, tet rule, near rule): the launch shape is
// a template parameter of the kernel, so each variant is its own instance.
struct VariantShape {
    int P;      // evaluation points per thread (block of 128 P points)
    int TILE;   // tets per pipeline stage (and per tile header)
    int S;      // pipeline stages
    int MINB;   // CTAs per SM the register budget is set for (__launch_bounds__)
    int DR;     // near-pair drain: routine called (0), inlined (1), inlined with the pair's state in shared memory (2),
                // or none (3): the near pairs are counted and left to the near pass
    int U;      // ray bundle: lines per lane per iteration of the ray rule
    bool PK;    // float32: packed registers pair two evaluation points (point-pair layout)
    int UJ;     // float32 far sweep: tet loop unrolled by UJ
};
using VariantLaunch = cudaError_t (*)(const VelocityArgs &a, int n_sm, cudaStream_t st, int *grid_out,
                                      bool query_only, int *occ_out);
struct VariantEntry {
    VariantShape s;
    VariantLaunch launch;
};
struct VariantList {
    const VariantEntry *v = nullptr;
    int n = 0;
};
// the instances, one translation unit per family (bs_vel_*.cu); n = 0 for an unsupported rule
VariantList variants_f32_q4();
VariantList variants_f32_rules(int Q);  // Q = 1, 8, 27, 64
VariantList variants_f64(int Q);
VariantList variants_exact(int precision, int Q);
VariantList velocity_variants(int precision, int Q, int near_rule);

constexpr int kMaxVariants = 32;  // num_variants() never exceeds this
int num_variants(int precision, int Q, int near_rule = BS_NEAR_RAY);
// the variant with one point per thread (128-point blocks) whose near pairs are drained in the far kernel
// (near_pass false) or left to a pass of their own (near_pass true), or -1: for meshes too small to fill the
// GPU with the default blocks
int small_mesh_variant(int precision, int Q, bool near_pass);
// the first variant that leaves the near pairs to a pass of their own (the near pass, or at the nodes the mesh
// walk), or -1
int near_pass_variant(int precision, int Q, int near_rule);
// a variant the fixed scratch of the no-alloc entry point can hold (quadrature-pair layout, tiles of 8..32
// tets), preferring one point per thread for the ray rule
int noalloc_variant(int precision, int Q, int near_rule);
constexpr int kSmallMeshWaves = 8;  // fewer default work items than this many GPU-fulls: a small mesh
// a batch of meshes of at most this many tets each takes the small-mesh variant (measured on 256 meshes of
// 8^3..24^3 nodes: 551 ms against 607 ms for the default variant)
constexpr int64_t kSmallBatchMeshTets = 80000;
LaunchShape shape_for(int precision, int Q, int variant = 0, int near_rule = 0);
int velocity_ctas_per_sm(int precision, int Q, int variant = 0, int near_rule = 0);
// ev_start/ev_stop (optional) are recorded around the velocity kernel alone
cudaError_t launch_velocity(int precision, const VelocityArgs &a, int n_sm, cudaStream_t st, int *grid_out,
                            cudaEvent_t ev_start = nullptr, cudaEvent_t ev_stop = nullptr);
cudaError_t launch_reduce(const VelocityArgs &a, cudaStream_t st);
// the near pass after the far sweep of a variant that leaves the near pairs to it (no-op otherwise); it returns
// at once when *a.near_skip is set (the mesh walk evaluated the near field)
cudaError_t launch_near_pass(int precision, const VelocityArgs &a, cudaStream_t st);
// autotuner cache (bs_tune.cu): key of a (GPU, precision, rule, near rule, directions, size class), the
// variant stored for it (-1 if none, or if its launch shape does not match the compiled variant table), and a store that
// also writes the cache file
std::string variant_shape_string(int precision, int Q, int near_rule, int variant);
std::string tune_key(const char *gpu_name, int n_sm, int precision, int Q, int near_rule, int L, int64_t k,
                     int64_t n_tets, bool at_nodes);
int tune_lookup(const std::string &key, int precision, int Q, int near_rule);
bool tune_store(const std::string &key, int precision, int Q, int near_rule, int variant, double ms, int candidates);
// all-ray kernel (bs_ray.cu): one point per thread, near records streamed in tiles of ray_shape().tile;
// single-mesh launches (a.meshes == nullptr); the partial sums and the reduction are those of the
// velocity kernel.  The float32 direction table is staged in shared memory: the host uses this kernel
// for tables of up to kRayLinesSmemMax lines only.
constexpr int kRayLinesSmemMax = 4096;
LaunchShape ray_shape();
int ray_ctas_per_sm(int precision, int L);
cudaError_t launch_ray(int precision, const VelocityArgs &a, int n_sm, cudaStream_t st, int *grid_out,
                       cudaEvent_t ev_start = nullptr, cudaEvent_t ev_stop = nullptr);

// Mesh walk (bs_walk.cu): the all-ray velocity at the mesh nodes by tracing every line through
// face neighbours.  Host-side connectivity, built once per handle from the tets:
struct WalkMesh {
    std::vector<int32_t> nbr;      // [n_tets][4] tet across the face opposite vertex i, or -1
    std::vector<int32_t> inc_off;  // [n_nodes + 1] CSR offsets of the node -> tet incidence
    std::vector<int32_t> inc;      // [4 n_tets] (tet << 2) | vertex index of the node in the tet
    std::vector<int32_t> bface;    // boundary faces as (tet << 2) | opposite vertex
    std::vector<int32_t> bnode;    // nodes on a boundary face
    bool conforming = false;       // every face shared by at most two tets, every node in some tet
};
bool build_walk_mesh(const int32_t *tets_host, int64_t n_nodes, int64_t n_tets, WalkMesh &w);
// Uniform grid of the boundary faces (device), for finding where a line re-enters a non-convex mesh.
struct WalkGrid {
    double lo[3], cell[3], inv[3];  // origin, cell size and its inverse per axis
    float lo32[3], cell32[3], inv32[3];  // the same in float (the float32 walk's search)
    int G;                          // cells per axis (G^3 cells)
    int ok;                         // 0 when the face lists overflowed their capacity
};
// Per boundary face (double, outward normal e1 x e2): vertex p0, edges e1, e2; and the face's (tet << 2) | face.
constexpr int kBFaceGeo = 9;
struct WalkGridArrays {
    WalkGrid *grid = nullptr;
    int32_t *cell_off = nullptr;   // [G^3 + 1]
    int32_t *cell_cnt = nullptr;   // [G^3] scratch
    int32_t *cell_face = nullptr;  // [cap] boundary-face indices
    double *geo = nullptr;         // [n_bface][kBFaceGeo]
    float *geo32 = nullptr;        // [n_bface][kBFaceGeo] float copy
    int G = 0;
    int64_t cap = 0;
};
struct WalkArgs {
    const double *nodes = nullptr;  // [n_nodes][3], also the evaluation points
    int64_t n_nodes = 0, n_tets = 0;
    const float4 *near32 = nullptr;
    const double *near64 = nullptr;
    const float4 *wrec = nullptr;  // float32 walk records [n_tets][kWalkRecVec4] (see bs_walk.cu)
    const int32_t *nbr = nullptr, *inc_off = nullptr, *inc = nullptr;
    const float4 *lines32 = nullptr;
    const dbl4 *lines64 = nullptr;
    int L = 0;
    double *out = nullptr;       // [n_nodes][3]
    int32_t *counts = nullptr;   // [n_nodes][3] or null
    // derivative of the velocity along directions e (the stretching term (omega . grad) v when e = omega):
    const double *omega = nullptr;  // [n_nodes][3] nodal vorticity (the directions when dirs is null)
    const double *dirs = nullptr;   // [n_nodes][3] or null
    double *dout = nullptr;         // [n_nodes][3] or null (no derivative)
    const int *mode = nullptr;   // device: 0 no walk, 1 walk (convex domain), 2 walk with re-entries
    const WalkGrid *grid = nullptr;
    const int32_t *cell_off = nullptr, *cell_face = nullptr, *bface = nullptr;
    const double *bgeo = nullptr;
    const float *bgeo32 = nullptr;
    int *flag = nullptr;
    int max_steps = 0;           // tets per half-line before the walk gives up (error flag)
    // near mode (the hybrid rule at the nodes): only the tets the far sweep's test calls near contribute
    // (pair_is_near_*, the same decision as the far sweep, which leaves them out), a half-line stops once it
    // is farther than *r_stop from the node (every tet beyond is far), warp w takes node perm[w] and writes
    // its totals to near_out[w] (float64, by spatial position) and its ray hits to counts[node][2]
    int near_mode = 0;
    const int *perm = nullptr;
    double *near_out = nullptr;
    const void *far = nullptr;        // far records (float32 tile frame, or float64)
    const float4 *tile_hdr = nullptr;
    int tile = 0, far_stride = 0;
    float far_ratio2_f = 0.f;
    double far_ratio2 = 0.0;
    const float *r_stop = nullptr;    // device: max over tets of far_ratio * circumradius + bounding radius
};
constexpr int kWalkRecVec4 = 8;  // float4 per float32 walk record (one 128-byte line)
// float32 walk records from the near records and the face neighbours (after every mesh update)
cudaError_t launch_walk_records(const float4 *near32, const int32_t *nbr, int64_t n_tets, float4 *wrec,
                                cudaStream_t st);
cudaError_t launch_walk_grid(const double *nodes, const int32_t *tets, const int32_t *bface, int64_t n_bface,
                             const int32_t *bnode, int64_t n_bnode, const WalkGridArrays &g, cudaStream_t st);
// after the convexity check and the grid: a non-convex mesh whose face grid overflowed gets mode 0
cudaError_t launch_walk_finalize(const WalkGrid *g, int *mode, cudaStream_t st);
// mode := 1 if conforming (else 0); 0 if two tets that share a face lie on the same side of it (a folded
// mesh); then 2 if a boundary node lies outside a boundary face's plane (a non-convex domain: the walk
// then looks for re-entries through the grid)
cudaError_t launch_convex_check(const double *nodes, const int32_t *tets, const int32_t *nbr, int64_t n_tets,
                                const int32_t *bface, int64_t n_bface, const int32_t *bnode, int64_t n_bnode,
                                float4 *bpos, int conforming, int *mode, float4 *wrec, cudaStream_t st);
cudaError_t launch_walk(int precision, const WalkArgs &a, cudaStream_t st, cudaEvent_t ev_start = nullptr,
                        cudaEvent_t ev_stop = nullptr);
// *r_stop := (1 + 1e-4) max over tets of (far_ratio * circumradius + bounding radius about the centroid):
// a half-line point farther than this from a node lies in no tet the node is near to
cudaError_t launch_near_reach(const double *rho2, const double *near64, int64_t n_tets, double far_ratio,
                              float *r_stop, cudaStream_t st);
// Heun step position updates (n_values = 3 * nodes)
cudaError_t launch_euler(const double *x0, const double *v0, double dt, int64_t n_values, double *x, cudaStream_t st);
cudaError_t launch_heun(const double *x0, const double *v0, const double *v1, double dt, int64_t n_values, double *x,
                        cudaStream_t st);

}  // namespace bs
