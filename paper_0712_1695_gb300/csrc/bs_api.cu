// bs_api.cu -- the C ABI of libbs (declared in include/bs.h): argument
// checks, device buffer ownership, table caching and kernel sequencing.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <cstring>

#include <algorithm>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "bs_internal.cuh"

using namespace bs;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    return fail(BS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define BS_CUDA(call)                                            \
    do {                                                         \
        cudaError_t _e = (call);                                 \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);      \
    } while (0)

bool valid_order(int q) { return q == 1 || q == 4 || q == 8 || q == 27 || q == 64; }

int check_params(const bs_params *p)
{
    if (!p) return fail(BS_ERR_ARG, "params is NULL");
    const double fr = p->far_ratio;
    if (isnan(fr) || (!isinf(fr) && fr < 2.0) || (isinf(fr) && fr < 0))
        return fail(BS_ERR_ARG, "far_ratio must be >= 2 or +INFINITY");
    if (p->n_theta < 1 || p->n_theta > 256 || p->n_phi < 1 || p->n_phi > 256)
        return fail(BS_ERR_ARG, "n_theta and n_phi must be in 1..256");
    if (p->precision != BS_FP32 && p->precision != BS_FP64) return fail(BS_ERR_ARG, "precision must be BS_FP64 or BS_FP32");
    if (!valid_order(p->tet_gauss_order)) return fail(BS_ERR_ORDER, "tet_gauss_order must be 1, 4, 8, 27 or 64");
    if (p->near_rule != BS_NEAR_RAY && p->near_rule != BS_NEAR_EXACT)
        return fail(BS_ERR_ARG, "near_rule must be BS_NEAR_RAY or BS_NEAR_EXACT");
    return BS_OK;
}

}  // namespace

// used by the other translation units of the library (bs_noalloc.cu)
void bs_set_last_error(const char *msg) { g_last_error = msg; }

struct bs_ctx {
    int device = 0;
    int n_sm = 0;
    int64_t n_nodes = 0, n_tets = 0;
    double *nodes = nullptr;
    int32_t *tets = nullptr;
    double *omega = nullptr;
    float4 *near32 = nullptr;
    double *near64 = nullptr;
    double *rho2 = nullptr;
    int *flag = nullptr;
    unsigned long long *first_bad = nullptr;
    unsigned long long *work_counter = nullptr;
    uint64_t version = 1;  // bumped whenever the near records change
    // far records of the last tet rule
    TetRule rule;
    uint64_t far_version = 0;
    float *far32 = nullptr;
    double *far64 = nullptr;
    float4 *tile_hdr = nullptr;
    int far_tile = 0;
    int far_layout = 0;            // float32 layout of far32 (kFarQuadPairs / kFarPointPairs)
    size_t far32_cap = 0, far64_cap = 0, hdr_cap = 0;  // allocated elements
    // spatial order of the evaluation points
    int *perm = nullptr;
    unsigned *keys = nullptr;
    size_t order_cap = 0;  // points
    int *cell_count = nullptr;
    int cell_bits = 0;
    int *box = nullptr;
    // direction table of the last (n_phi, n_theta)
    LineTables lines;
    // scratch for per-chunk partial sums, and the near pass's totals ([k][3], variants that take it)
    double *partial = nullptr;
    size_t partial_cap = 0;
    double *near_out = nullptr;
    size_t near_cap = 0;
    float *r_stop = nullptr;  // the near walk's stop radius (device), for rstop_version and rstop_fr
    uint64_t rstop_version = 0;
    double rstop_fr = 0.0;
    // staging for bs_velocity_host
    double *stage = nullptr;
    size_t stage_cap = 0;
    // work arrays of bs_rk2_step: x0, v0, v1 (each [n_nodes][3]); of bs_rk2_step_stretch also w0, s0, s1
    double *rk = nullptr;
    double *rk_w = nullptr;
    int occ[2][2][65][kMaxVariants] = {};  // cached CTAs per SM by [near rule][precision][Q][variant]
    int ray_occ[2] = {};                   // cached CTAs per SM of the all-ray kernel by [precision]
    int ray_occ_L[2] = {};                 // ... for this many directions
    int pinned[2][2][65];                  // bs_set_variant by [near rule][precision][Q], -1: automatic
    int tuned[2][2][2][65] = {};           // the variant bs_autotune last chose (or found in the cache) by
                                           // [nodes path][near rule][precision][Q]
    std::map<std::string, int> tune_memo;  // tuning key -> cached variant (-1: no entry)
    char gpu_name[256] = {};
    // mesh walk of the all-ray velocity at the nodes (built on first use)
    bool walk_built = false;
    bool walk_conforming = false;
    int32_t *walk_nbr = nullptr, *walk_inc_off = nullptr, *walk_inc = nullptr, *walk_bface = nullptr,
            *walk_bnode = nullptr;
    int64_t walk_n_bface = 0, walk_n_bnode = 0;
    int *walk_mode = nullptr;      // device: the walk is valid for the current node positions
    float4 *walk_rec = nullptr;    // float32 walk records [n_tets][kWalkRecVec4]
    float4 *walk_bpos = nullptr;   // convexity check work array [2 n_bnode + 1]
    WalkGridArrays walk_grid;      // boundary faces on a uniform grid (re-entries into a non-convex mesh)
    uint64_t walk_version = 0;     // mesh version when walk_mode was computed
    // bs_rk2_steps: a stream of the handle on which steps are captured and replayed as a CUDA graph, and
    // the events that join it to the caller's stream
    cudaStream_t step_stream = nullptr;
    cudaEvent_t step_in = nullptr, step_out = nullptr;
    int64_t graph_steps = 0;  // steps run by graph replay since the handle was created
    // kernel timing (bs_profile)
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used, ev_free;
    int64_t prof_kernel = 0, prof_all = 0;
    // bounded-wait settings (bs_set_wait_limits): 0 = the defaults
    int64_t walk_max_steps = 0;
    int64_t copy_wait_polls = 0;
    int withhold_copies = 0;
};

namespace {

void drop_events(bs_ctx *h)
{
    for (auto &p : h->ev_used) h->ev_free.push_back(p);
    h->ev_used.clear();
}

void free_ctx(bs_ctx *h)
{
    drop_events(h);
    if (h->step_in) cudaEventDestroy(h->step_in);
    if (h->step_out) cudaEventDestroy(h->step_out);
    if (h->step_stream) cudaStreamDestroy(h->step_stream);
    for (auto &p : h->ev_free) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    void *bufs[] = {h->nodes, h->tets,  h->omega,     h->near32,   h->near64,  h->rho2,         h->flag,
                    h->first_bad, h->work_counter, h->rule.bary, h->rule.w, h->far32, h->far64, h->lines.f32,
                    h->lines.f64, h->partial, h->stage, h->rk, h->tile_hdr, h->perm, h->keys,
                    h->cell_count, h->box, h->walk_nbr, h->walk_inc_off, h->walk_inc, h->walk_bface,
                    h->walk_bnode, h->walk_mode, h->walk_rec, h->walk_bpos, h->rk_w, h->walk_grid.grid,
                    h->walk_grid.cell_off, h->walk_grid.cell_cnt, h->walk_grid.cell_face, h->walk_grid.geo,
                    h->walk_grid.geo32, h->near_out, h->r_stop};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete h;
}

}  // namespace

struct bs_batch_ctx {
    std::vector<bs_ctx *> meshes;
    int device = 0, n_sm = 0;
    std::vector<int64_t> point_begin;
    int64_t n_points = 0;
    std::vector<uint64_t> order_version;  // mesh version when its point order was computed
    int *perm = nullptr;                  // [n_points] per-mesh visiting orders, concatenated
    unsigned *keys = nullptr;
    int *cell_count = nullptr;
    int cell_bits = 0;
    int *box = nullptr;
    MeshDesc *d_meshes = nullptr;
    std::vector<MeshDesc> h_meshes;  // last descriptor table copied to the device
    double *partial = nullptr;
    size_t partial_cap = 0;
    double *near_out = nullptr;  // the near pass's totals over all meshes' points
    std::vector<WalkArgs> walks;  // per mesh: the near walk of the captured launch sequence (empty: none)
    // the near walks run concurrently on side streams, forked from the caller's stream and joined back into it
    std::vector<cudaStream_t> walk_streams;
    std::vector<cudaEvent_t> walk_events;  // [0] the fork, [1 + k] the join of side stream k
    const int **d_near_skip = nullptr;   // device [n]: per mesh, the walk's mode flag (near pass skips walked meshes)
    std::vector<const int *> h_near_skip;  // its host copy
    unsigned long long *work_counter = nullptr;
    int *flag = nullptr;
    LineTables lines;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    int graph_prec = -1;
    VelocityArgs graph_args;
};

namespace {

void free_batch(bs_batch_ctx *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaStream_t s : b->walk_streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->walk_events) cudaEventDestroy(e);
    void *bufs[] = {b->perm, b->keys, b->cell_count, b->box, b->d_meshes, b->partial, b->work_counter, b->flag,
                    b->lines.f32, b->lines.f64, b->near_out, (void *)b->d_near_skip};
    for (void *p : bufs)
        if (p) cudaFree(p);
    delete b;
}

cudaError_t ensure_lines(bs_ctx *h, int n_phi, int n_theta, cudaStream_t st)
{
    if (h->lines.f32 && h->lines.n_phi == n_phi && h->lines.n_theta == n_theta) return cudaSuccess;
    if (h->lines.f32) cudaFreeAsync(h->lines.f32, st);
    if (h->lines.f64) cudaFreeAsync(h->lines.f64, st);
    h->lines = LineTables();
    const size_t L = (size_t)n_phi * n_theta;
    cudaError_t e = cudaMallocAsync((void **)&h->lines.f32, L * sizeof(float4), st);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync((void **)&h->lines.f64, L * sizeof(dbl4), st);
    if (e != cudaSuccess) return e;
    e = build_lines(n_phi, n_theta, h->lines.f32, h->lines.f64, st);
    if (e != cudaSuccess) return e;
    if (h->prof) h->prof_all += 1;
    h->lines.n_phi = n_phi;
    h->lines.n_theta = n_theta;
    return cudaSuccess;
}

// The far records of tet rule Q in the float32 layout and tile size of the variant a call uses (the tile
// headers and the float32 tile frame depend on the tile), rebuilt when the mesh changed.
cudaError_t ensure_far(bs_ctx *h, int Q, int tile, int layout, cudaStream_t st)
{
    if (h->far32 && h->rule.order == Q && h->far_tile == tile && h->far_layout == layout &&
        h->far_version == h->version)
        return cudaSuccess;
    cudaError_t e;
    if (h->rule.order != Q) {
        if (h->rule.bary) cudaFreeAsync(h->rule.bary, st);
        if (h->rule.w) cudaFreeAsync(h->rule.w, st);
        h->rule = TetRule();
        if ((e = cudaMallocAsync((void **)&h->rule.bary, sizeof(double) * 4 * Q, st)) != cudaSuccess) return e;
        if ((e = cudaMallocAsync((void **)&h->rule.w, sizeof(double) * Q, st)) != cudaSuccess) return e;
        if ((e = build_tet_rule(Q, h->rule.bary, h->rule.w, st)) != cudaSuccess) return e;
        if (h->prof) h->prof_all += 1;
        h->rule.order = Q;
    }
    const size_t n = (size_t)std::max<int64_t>(h->n_tets, 1);
    auto grow = [&](void **buf, size_t &cap, size_t need, size_t elem) -> cudaError_t {
        if (need <= cap && *buf) return cudaSuccess;
        if (*buf) cudaFreeAsync(*buf, st);
        *buf = nullptr;
        cap = 0;
        cudaError_t r = cudaMallocAsync(buf, need * elem, st);
        if (r == cudaSuccess) cap = need;
        return r;
    };
    if ((e = grow((void **)&h->far32, h->far32_cap, n * far_stride<float>(Q, layout), sizeof(float))) != cudaSuccess)
        return e;
    if ((e = grow((void **)&h->far64, h->far64_cap, n * far_stride<double>(Q), sizeof(double))) != cudaSuccess)
        return e;
    if ((e = grow((void **)&h->tile_hdr, h->hdr_cap, 2 * ((n + tile - 1) / tile), sizeof(float4))) != cudaSuccess)
        return e;
    if ((e = build_far_records(h->near64, h->rho2, h->n_tets, h->rule, tile, layout, h->tile_hdr, h->far32, h->far64,
                               st)) != cudaSuccess)
        return e;
    if (h->prof) h->prof_all += 2;
    h->far_tile = tile;
    h->far_layout = layout;
    h->far_version = h->version;
    return cudaSuccess;
}

// The kernel variant of the velocity kernel a call on k points uses: the environment variable
// BS_VARIANT, else the variant bs_set_variant pinned, else the autotuner's cache entry for this GPU and
// problem (at_nodes: the mesh's nodes by bs_velocity_nodes, where the walk can take the near field), else,
// for the ray rule: at the nodes (directions within the walk's table) a variant that leaves the near pairs to
// the walk -- with one point per thread on a small mesh -- and elsewhere, on a small mesh, the one-point
// variant that drains them in the far kernel; else variant 0.
int choose_variant(bs_ctx *h, const bs_params *p, int64_t k, bool at_nodes)
{
    const int prec = p->precision, Q = p->tet_gauss_order, nr = p->near_rule;
    const int nv = num_variants(prec, Q, nr);
    const char *env = getenv("BS_VARIANT");
    if (env) {
        const int v = atoi(env);
        return (v >= 0 && v < nv) ? v : 0;
    }
    const int pin = h->pinned[nr][prec][Q];
    if (pin >= 0 && pin < nv) return pin;
    const std::string key =
        tune_key(h->gpu_name, h->n_sm, prec, Q, nr, p->n_phi * p->n_theta, k, h->n_tets, at_nodes);
    auto it = h->tune_memo.find(key);
    const int tv = it != h->tune_memo.end() ? it->second : (h->tune_memo[key] = tune_lookup(key, prec, Q, nr));
    if (tv >= 0 && tv < nv) return tv;
    if (nr == BS_NEAR_RAY) {
        // a mesh whose default work items would not fill the GPU several times over: 128-point blocks give
        // it three times as many warps (for the in-kernel drain, three times as many warps draining near pairs)
        auto small = [&]() {
            const LaunchShape s0 = shape_for(prec, Q, 0, nr);
            int &o0 = h->occ[nr][prec][Q][0];
            if (o0 == 0) o0 = std::max(1, velocity_ctas_per_sm(prec, Q, 0, nr));
            const int64_t b0 = (k + (int64_t)s0.threads * s0.points_per_thread - 1) /
                               ((int64_t)s0.threads * s0.points_per_thread);
            const int64_t t0 = (h->n_tets + s0.tile - 1) / s0.tile;
            return b0 * ((t0 + kMinTilesPerItem - 1) / kMinTilesPerItem) < (int64_t)kSmallMeshWaves * h->n_sm * o0;
        };
        // at the nodes the walk's cost grows with the chords it integrates, the in-kernel drain's with every
        // line of every near pair: leave the near pairs to the walk
        if (at_nodes && p->n_phi * p->n_theta <= kRayLinesSmemMax) {
            const int sv = small_mesh_variant(prec, Q, true);
            if (sv >= 0 && small()) return sv;
            const int dv = near_pass_variant(prec, Q, nr);
            if (dv >= 0) return dv;
        } else {
            const int sv = small_mesh_variant(prec, Q, false);
            if (sv >= 0 && small()) return sv;
        }
    }
    return 0;
}

cudaError_t ensure_order(bs_ctx *h, int64_t k, int bits, cudaStream_t st)
{
    cudaError_t e;
    if ((size_t)k > h->order_cap) {
        if (h->perm) cudaFreeAsync(h->perm, st);
        if (h->keys) cudaFreeAsync(h->keys, st);
        h->perm = nullptr;
        h->keys = nullptr;
        h->order_cap = 0;
        if ((e = cudaMallocAsync((void **)&h->perm, sizeof(int) * k, st)) != cudaSuccess) return e;
        if ((e = cudaMallocAsync((void **)&h->keys, sizeof(unsigned) * k, st)) != cudaSuccess) return e;
        h->order_cap = (size_t)k;
    }
    if (bits > h->cell_bits) {
        if (h->cell_count) cudaFreeAsync(h->cell_count, st);
        h->cell_count = nullptr;
        h->cell_bits = 0;
        if ((e = cudaMallocAsync((void **)&h->cell_count, sizeof(int) << (3 * bits), st)) != cudaSuccess) return e;
        h->cell_bits = bits;
    }
    if (!h->box && (e = cudaMallocAsync((void **)&h->box, sizeof(int) * 8, st)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t ensure_partial(bs_ctx *h, size_t bytes, cudaStream_t st)
{
    if (bytes <= h->partial_cap) return cudaSuccess;
    if (h->partial) cudaFreeAsync(h->partial, st);
    h->partial = nullptr;
    h->partial_cap = 0;
    cudaError_t e = cudaMallocAsync((void **)&h->partial, bytes, st);
    if (e == cudaSuccess) h->partial_cap = bytes;
    return e;
}

}  // namespace

extern "C" {

const char *bs_last_error(void) { return g_last_error.c_str(); }

int bs_create(const double *nodes, int64_t n_nodes, const int32_t *tets, int64_t n_tets, const double *omega,
              bs_handle *out)
{
    if (!out) return fail(BS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!nodes || !omega || (n_tets > 0 && !tets)) return fail(BS_ERR_ARG, "NULL mesh array");
    if (n_nodes < 1 || n_tets < 0) return fail(BS_ERR_ARG, "need n_nodes >= 1 and n_tets >= 0");
    if (n_nodes > INT32_MAX) return fail(BS_ERR_ARG, "n_nodes exceeds the int32 index range");
    bs_ctx *h = new bs_ctx();
    h->n_nodes = n_nodes;
    h->n_tets = n_tets;
    for (auto &a : h->pinned)
        for (auto &b : a)
            for (int &c : b) c = -1;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
    cudaDeviceProp prop;
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, h->device);
    if (e == cudaSuccess) snprintf(h->gpu_name, sizeof h->gpu_name, "%s", prop.name);
    const size_t nt = (size_t)std::max<int64_t>(n_tets, 1);
    if (e == cudaSuccess) e = cudaMalloc(&h->nodes, sizeof(double) * 3 * n_nodes);
    if (e == cudaSuccess) e = cudaMalloc(&h->omega, sizeof(double) * 3 * n_nodes);
    if (e == cudaSuccess) e = cudaMalloc(&h->tets, sizeof(int32_t) * 4 * nt);
    if (e == cudaSuccess) e = cudaMalloc(&h->near32, sizeof(float4) * kNearF32Vec4 * nt);
    if (e == cudaSuccess) e = cudaMalloc(&h->near64, sizeof(double) * kNearF64 * nt);
    if (e == cudaSuccess) e = cudaMalloc(&h->rho2, sizeof(double) * nt);
    if (e == cudaSuccess) e = cudaMalloc(&h->flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->first_bad, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&h->work_counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(h->nodes, nodes, sizeof(double) * 3 * n_nodes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->omega, omega, sizeof(double) * 3 * n_nodes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_tets > 0)
        e = cudaMemcpy(h->tets, tets, sizeof(int32_t) * 4 * n_tets, cudaMemcpyHostToDevice);
    const unsigned long long none = ~0ull;
    if (e == cudaSuccess) e = cudaMemset(h->flag, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(h->first_bad, &none, sizeof(none), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = build_near_records(h->nodes, n_nodes, h->tets, n_tets, h->omega, h->near32, h->near64, h->rho2, h->flag,
                               h->first_bad, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int flag = 0;
    unsigned long long bad = none;
    if (e == cudaSuccess) e = cudaMemcpy(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&bad, h->first_bad, sizeof(bad), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        free_ctx(h);
        return cuda_fail(e, "bs_create");
    }
    if (flag) {
        free_ctx(h);
        char msg[160];
        snprintf(msg, sizeof msg, "tet %llu: %s", bad,
                 (flag & kFlagMeshIndex) ? "node index out of range (or degenerate tet)"
                                         : "degenerate tet (|volume| <= 1e-14 h^3)");
        return fail(BS_ERR_MESH, msg);
    }
    *out = h;
    return BS_OK;
}

int bs_update(bs_handle h, const double *nodes_dev, const double *omega_dev, void *stream)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (nodes_dev)
        BS_CUDA(cudaMemcpyAsync(h->nodes, nodes_dev, sizeof(double) * 3 * h->n_nodes, cudaMemcpyDeviceToDevice, st));
    if (omega_dev)
        BS_CUDA(cudaMemcpyAsync(h->omega, omega_dev, sizeof(double) * 3 * h->n_nodes, cudaMemcpyDeviceToDevice, st));
    BS_CUDA(build_near_records(h->nodes, h->n_nodes, h->tets, h->n_tets, h->omega, h->near32, h->near64, h->rho2,
                               h->flag, h->first_bad, st));
    if (h->prof && h->n_tets > 0) h->prof_all += 1;
    ++h->version;
    return BS_OK;
}

int bs_rk2_step(bs_handle h, double dt, const bs_params *p, void *stream)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->counts) return fail(BS_ERR_ARG, "bs_rk2_step: counts are not supported (set p->counts = NULL)");
    if (!std::isfinite(dt)) return fail(BS_ERR_ARG, "bs_rk2_step: dt must be finite");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = h->n_nodes, nv = 3 * n;
    if (!h->rk) BS_CUDA(cudaMallocAsync((void **)&h->rk, sizeof(double) * 3 * nv, st));
    double *x0 = h->rk, *v0 = h->rk + nv, *v1 = h->rk + 2 * nv;
    BS_CUDA(cudaMemcpyAsync(x0, h->nodes, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
    if ((rc = bs_velocity_nodes(h, p, v0, stream))) return rc;
    BS_CUDA(launch_euler(x0, v0, dt, nv, h->nodes, st));  // the mesh moves to x*
    if ((rc = bs_update(h, nullptr, nullptr, stream))) return rc;
    if ((rc = bs_velocity_nodes(h, p, v1, stream))) return rc;
    BS_CUDA(launch_heun(x0, v0, v1, dt, nv, h->nodes, st));  // and on to x1
    if ((rc = bs_update(h, nullptr, nullptr, stream))) return rc;
    if (h->prof) h->prof_all += 2;
    return BS_OK;
}

int bs_omega(bs_handle h, double *omega_dev, void *stream)
{
    if (!h || !omega_dev) return fail(BS_ERR_ARG, "NULL argument");
    BS_CUDA(cudaMemcpyAsync(omega_dev, h->omega, sizeof(double) * 3 * h->n_nodes, cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
    return BS_OK;
}

int bs_nodes(bs_handle h, double *nodes_dev, void *stream)
{
    if (!h || !nodes_dev) return fail(BS_ERR_ARG, "NULL argument");
    BS_CUDA(cudaMemcpyAsync(nodes_dev, h->nodes, sizeof(double) * 3 * h->n_nodes, cudaMemcpyDeviceToDevice,
                            (cudaStream_t)stream));
    return BS_OK;
}

int bs_status(bs_handle h, void *stream)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    BS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int flag = 0;
    BS_CUDA(cudaMemcpy(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost));
    BS_CUDA(cudaMemset(h->flag, 0, sizeof(int)));
    if (flag & kFlagTimeout) return fail(BS_ERR_TIMEOUT, "a bounded device wait gave up");
    if (flag & kFlagWalk) return fail(BS_ERR_TIMEOUT, "a mesh walk did not leave the mesh within its step limit");
    if (flag & kFlagWalkStuck) return fail(BS_ERR_MESH, "a mesh walk reached a tet with no face ahead of the line");
    if (flag & kFlagNoWalk)
        return fail(BS_ERR_MESH, "the derivative along directions needs a conforming mesh with a convex domain "
                                 "(the mesh walk); the velocity was computed, the derivative was not");
    if (flag & (kFlagMeshIndex | kFlagMeshVolume)) return fail(BS_ERR_MESH, "degenerate tet after bs_update");
    return BS_OK;
}

int bs_set_wait_limits(bs_handle h, int64_t walk_max_steps, int64_t copy_wait_polls, int withhold_copies)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    if (walk_max_steps < 0 || copy_wait_polls < 0 || (withhold_copies != 0 && withhold_copies != 1))
        return fail(BS_ERR_ARG, "bs_set_wait_limits: limits must be >= 0 and withhold_copies 0 or 1");
    h->walk_max_steps = walk_max_steps;
    h->copy_wait_polls = copy_wait_polls;
    h->withhold_copies = withhold_copies;
    return BS_OK;
}

int bs_mesh_size(bs_handle h, int64_t *n_nodes, int64_t *n_tets)
{
    if (!h || !n_nodes || !n_tets) return fail(BS_ERR_ARG, "NULL argument");
    *n_nodes = h->n_nodes;
    *n_tets = h->n_tets;
    return BS_OK;
}

namespace {
int velocity_impl(bs_handle h, const double *eval_pts_dev, int64_t k, const bs_params *p, double *out_dev,
                  void *stream, const int *skip, const WalkArgs *near_walk = nullptr);
}

int bs_velocity(bs_handle h, const double *eval_pts_dev, int64_t k, const bs_params *p, double *out_dev,
                void *stream)
{
    return velocity_impl(h, eval_pts_dev, k, p, out_dev, stream, nullptr);
}

namespace {

// The mesh walk's connectivity (host build, synchronous, once per handle) and device arrays.
cudaError_t ensure_walk(bs_ctx *h)
{
    if (h->walk_built) return cudaSuccess;
    std::vector<int32_t> tets((size_t)4 * h->n_tets);
    cudaError_t e = cudaMemcpy(tets.data(), h->tets, sizeof(int32_t) * tets.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    WalkMesh w;
    build_walk_mesh(tets.data(), h->n_nodes, h->n_tets, w);
    auto up = [](int32_t **dst, const std::vector<int32_t> &v) -> cudaError_t {
        cudaError_t r = cudaMalloc((void **)dst, sizeof(int32_t) * std::max<size_t>(v.size(), 1));
        if (r != cudaSuccess || v.empty()) return r;
        return cudaMemcpy(*dst, v.data(), sizeof(int32_t) * v.size(), cudaMemcpyHostToDevice);
    };
    if ((e = up(&h->walk_nbr, w.nbr)) != cudaSuccess) return e;
    if ((e = up(&h->walk_inc_off, w.inc_off)) != cudaSuccess) return e;
    if ((e = up(&h->walk_inc, w.inc)) != cudaSuccess) return e;
    if ((e = up(&h->walk_bface, w.bface)) != cudaSuccess) return e;
    if ((e = up(&h->walk_bnode, w.bnode)) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&h->walk_mode, sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&h->walk_rec, sizeof(float4) * kWalkRecVec4 * std::max<int64_t>(h->n_tets, 1))) !=
        cudaSuccess)
        return e;
    h->walk_n_bface = (int64_t)w.bface.size();
    h->walk_n_bnode = (int64_t)w.bnode.size();
    if ((e = cudaMalloc((void **)&h->walk_bpos, sizeof(float4) * (2 * h->walk_n_bnode + 1))) != cudaSuccess) return e;
    // face grid: the boundary is a surface, about 6 G^2 of the G^3 cells hold its faces; G for a few faces per
    // surface cell; lists of up to 16 cells per face
    WalkGridArrays &g = h->walk_grid;
    g.G = (int)std::min<double>(160.0, std::max(4.0, std::round(std::sqrt((double)h->walk_n_bface / 8.0))));
    const int64_t cells = (int64_t)g.G * g.G * g.G;
    g.cap = 16 * std::max<int64_t>(h->walk_n_bface, 1);
    if ((e = cudaMalloc((void **)&g.grid, sizeof(WalkGrid))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&g.cell_off, sizeof(int32_t) * (cells + 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&g.cell_cnt, sizeof(int32_t) * cells)) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&g.cell_face, sizeof(int32_t) * g.cap)) != cudaSuccess) return e;
    if ((e = cudaMalloc((void **)&g.geo, sizeof(double) * kBFaceGeo * std::max<int64_t>(h->walk_n_bface, 1))) !=
        cudaSuccess)
        return e;
    if ((e = cudaMalloc((void **)&g.geo32, sizeof(float) * kBFaceGeo * std::max<int64_t>(h->walk_n_bface, 1))) !=
        cudaSuccess)
        return e;
    h->walk_conforming = w.conforming && 4 * h->n_tets < INT32_MAX;
    h->walk_built = true;
    h->walk_version = 0;
    return cudaSuccess;
}

}  // namespace

namespace {

// The walk's tables for the current node positions: face adjacency (first use), then, after every change of
// the nodes, the walk records, the convexity and fold checks and the boundary-face grid (all queued on st).
cudaError_t walk_prepare(bs_ctx *h, cudaStream_t st)
{
    cudaError_t e = ensure_walk(h);
    if (e != cudaSuccess || h->walk_version == h->version) return e;
    if ((e = launch_walk_records(h->near32, h->walk_nbr, h->n_tets, h->walk_rec, st)) != cudaSuccess) return e;
    if ((e = launch_convex_check(h->nodes, h->tets, h->walk_nbr, h->n_tets, h->walk_bface, h->walk_n_bface,
                                 h->walk_bnode, h->walk_n_bnode, h->walk_bpos, h->walk_conforming ? 1 : 0,
                                 h->walk_mode, h->walk_rec, st)) != cudaSuccess)
        return e;
    if (h->walk_conforming) {
        if ((e = launch_walk_grid(h->nodes, h->tets, h->walk_bface, h->walk_n_bface, h->walk_bnode, h->walk_n_bnode,
                                  h->walk_grid, st)) != cudaSuccess)
            return e;
        if ((e = launch_walk_finalize(h->walk_grid.grid, h->walk_mode, st)) != cudaSuccess) return e;
        if (h->prof) h->prof_all += 5;
    }
    h->walk_version = h->version;
    if (h->prof)
        h->prof_all += 2 + (h->walk_conforming && h->n_tets > 0 ? 1 : 0) +
                       (h->walk_conforming && h->walk_n_bface > 0 && h->walk_n_bnode > 0 ? 2 : 0);
    return cudaSuccess;
}

// the walk's arguments that come from the mesh handle (tables, flags, step limit)
void walk_args(bs_ctx *h, WalkArgs &w)
{
    w.nodes = h->nodes;
    w.n_nodes = h->n_nodes;
    w.n_tets = h->n_tets;
    w.near32 = h->near32;
    w.near64 = h->near64;
    w.wrec = h->walk_rec;
    w.nbr = h->walk_nbr;
    w.inc_off = h->walk_inc_off;
    w.inc = h->walk_inc;
    w.omega = h->omega;
    w.mode = h->walk_mode;
    w.grid = h->walk_grid.grid;
    w.cell_off = h->walk_grid.cell_off;
    w.cell_face = h->walk_grid.cell_face;
    w.bface = h->walk_bface;
    w.bgeo = h->walk_grid.geo;
    w.bgeo32 = h->walk_grid.geo32;
    w.flag = h->flag;
    // no valid mesh needs more steps than tets; a small cap keeps a broken walk short
    w.max_steps = (int)std::min<int64_t>(h->n_tets, std::max<int64_t>(4096, 64 * (int64_t)std::cbrt((double)h->n_tets)));
    if (h->walk_max_steps > 0) w.max_steps = (int)std::min<int64_t>(h->walk_max_steps, INT32_MAX);
}

// the near walk's stop radius for the mesh's current version and the far ratio
cudaError_t ensure_rstop(bs_ctx *h, double far_ratio, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    if (!h->r_stop && (e = cudaMallocAsync((void **)&h->r_stop, sizeof(float), st)) != cudaSuccess) return e;
    if (h->rstop_version != h->version || h->rstop_fr != far_ratio) {
        if ((e = launch_near_reach(h->rho2, h->near64, h->n_tets, far_ratio, h->r_stop, st)) != cudaSuccess) return e;
        h->rstop_version = h->version;
        h->rstop_fr = far_ratio;
        if (h->prof) h->prof_all += 1;
    }
    return cudaSuccess;
}

// Velocity at the nodes (and, with dout, its derivative along dirs or the nodal vorticity): the mesh walk
// in all-ray mode, else bs_velocity at the nodes.
int nodes_impl(bs_handle h, const bs_params *p, double *out_dev, const double *dirs, double *dout, void *stream)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    int rc = check_params(p);
    if (rc) return rc;
    if (!out_dev) return fail(BS_ERR_ARG, "NULL output");
    const int L = p->n_phi * p->n_theta;
    const char *env = getenv("BS_WALK");
    const bool can_walk = L <= kRayLinesSmemMax && h->n_tets > 0 && !(env && atoi(env) == 0) &&
                          p->near_rule == BS_NEAR_RAY;
    const bool walk = isinf(p->far_ratio) && can_walk;  // the all-ray rule at every pair
    if (dout && !walk)
        return fail(BS_ERR_ARG, "the derivative along directions is the all-ray method's (far_ratio = +inf, at most "
                                "4096 directions) computed by the mesh walk");
    // the hybrid rule: the walk takes the near field when the variant leaves it to a pass of its own
    const bool near_walk = !isinf(p->far_ratio) && can_walk && !dout &&
                           shape_for(p->precision, p->tet_gauss_order, choose_variant(h, p, h->n_nodes, true),
                                     p->near_rule).drain == 3;
    if (!walk && !near_walk) return velocity_impl(h, h->nodes, h->n_nodes, p, out_dev, stream, nullptr);
    cudaStream_t st = (cudaStream_t)stream;
    BS_CUDA(walk_prepare(h, st));
    BS_CUDA(ensure_lines(h, p->n_phi, p->n_theta, st));
    WalkArgs w;
    walk_args(h, w);
    w.lines32 = h->lines.f32;
    w.lines64 = h->lines.f64;
    w.L = L;
    w.out = out_dev;
    w.counts = p->counts;
    w.dirs = dirs;
    w.dout = dout;
    if (near_walk) {
        // the stop radius for this mesh version and far ratio; velocity_impl fills in the rest
        BS_CUDA(ensure_rstop(h, p->far_ratio, st));
        w.near_mode = 1;
        w.r_stop = h->r_stop;
        w.counts = p->counts;
        return velocity_impl(h, h->nodes, h->n_nodes, p, out_dev, stream, nullptr, &w);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->prof) {
        if (h->ev_free.empty()) {
            BS_CUDA(cudaEventCreate(&e0));
            BS_CUDA(cudaEventCreate(&e1));
        } else {
            e0 = h->ev_free.back().first;
            e1 = h->ev_free.back().second;
            h->ev_free.pop_back();
        }
        h->ev_used.push_back({e0, e1});
        h->prof_kernel += 1;
        h->prof_all += 1;
    }
    BS_CUDA(launch_walk(p->precision, w, st, e0, e1));
    // the all-ray kernel for a domain the walk cannot serve (returns at once otherwise)
    const bool prof = h->prof;
    h->prof = false;  // the walk's events time this call
    rc = velocity_impl(h, h->nodes, h->n_nodes, p, out_dev, stream, h->walk_mode);
    h->prof = prof;
    if (prof) h->prof_all += 5 + 3;
    return rc;
}

}  // namespace

int bs_velocity_nodes(bs_handle h, const bs_params *p, double *out_dev, void *stream)
{
    return nodes_impl(h, p, out_dev, nullptr, nullptr, stream);
}

int bs_velocity_nodes_dderiv(bs_handle h, const bs_params *p, const double *dirs_dev, double *out_dev,
                             double *dout_dev, void *stream)
{
    if (!dout_dev) return fail(BS_ERR_ARG, "NULL derivative output");
    return nodes_impl(h, p, out_dev, dirs_dev, dout_dev, stream);
}

int bs_rk2_step_stretch(bs_handle h, double dt, const bs_params *p, void *stream)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->counts) return fail(BS_ERR_ARG, "bs_rk2_step_stretch: counts are not supported (set p->counts = NULL)");
    if (!std::isfinite(dt)) return fail(BS_ERR_ARG, "bs_rk2_step_stretch: dt must be finite");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = h->n_nodes, nv = 3 * n;
    if (!h->rk) BS_CUDA(cudaMallocAsync((void **)&h->rk, sizeof(double) * 3 * nv, st));
    if (!h->rk_w) BS_CUDA(cudaMallocAsync((void **)&h->rk_w, sizeof(double) * 3 * nv, st));
    double *x0 = h->rk, *v0 = h->rk + nv, *v1 = h->rk + 2 * nv;
    double *w0 = h->rk_w, *s0 = h->rk_w + nv, *s1 = h->rk_w + 2 * nv;
    BS_CUDA(cudaMemcpyAsync(x0, h->nodes, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
    BS_CUDA(cudaMemcpyAsync(w0, h->omega, sizeof(double) * nv, cudaMemcpyDeviceToDevice, st));
    // stage 1: v0 and the stretching s0 = (omega . grad) v at (x0, w0)
    if ((rc = nodes_impl(h, p, v0, nullptr, s0, stream))) return rc;
    BS_CUDA(launch_euler(x0, v0, dt, nv, h->nodes, st));  // x* = x0 + dt v0
    BS_CUDA(launch_euler(w0, s0, dt, nv, h->omega, st));  // w* = w0 + dt s0
    if ((rc = bs_update(h, nullptr, nullptr, stream))) return rc;
    // stage 2 at (x*, w*), then the Heun average
    if ((rc = nodes_impl(h, p, v1, nullptr, s1, stream))) return rc;
    BS_CUDA(launch_heun(x0, v0, v1, dt, nv, h->nodes, st));
    BS_CUDA(launch_heun(w0, s0, s1, dt, nv, h->omega, st));
    if ((rc = bs_update(h, nullptr, nullptr, stream))) return rc;
    if (h->prof) h->prof_all += 4;
    return BS_OK;
}

int bs_rk2_steps(bs_handle h, double dt, int64_t n_steps, int stretch, const bs_params *p, void *stream)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    if (n_steps < 0) return fail(BS_ERR_ARG, "bs_rk2_steps: n_steps < 0");
    if (stretch != 0 && stretch != 1) return fail(BS_ERR_ARG, "bs_rk2_steps: stretch must be 0 or 1");
    int rc = check_params(p);
    if (rc) return rc;
    if (n_steps == 0) return BS_OK;
    auto step = [&](void *s) { return stretch ? bs_rk2_step_stretch(h, dt, p, s) : bs_rk2_step(h, dt, p, s); };
    // the first step runs as it is: it allocates the work arrays and builds what the later steps reuse
    if ((rc = step(stream))) return rc;
    int64_t done = 1;
    if (n_steps > 1 && !h->prof) {  // under bs_profile every launch is counted, so the steps run one by one
        cudaStream_t caller = (cudaStream_t)stream;
        if (!h->step_stream) {
            BS_CUDA(cudaStreamCreateWithFlags(&h->step_stream, cudaStreamNonBlocking));
            BS_CUDA(cudaEventCreateWithFlags(&h->step_in, cudaEventDisableTiming));
            BS_CUDA(cudaEventCreateWithFlags(&h->step_out, cudaEventDisableTiming));
        }
        cudaStream_t ss = h->step_stream;
        BS_CUDA(cudaEventRecord(h->step_in, caller));
        BS_CUDA(cudaStreamWaitEvent(ss, h->step_in, 0));
        // capture one step.  It launches the same kernels with the same arguments as the eager step: the
        // handle's buffers are all allocated by now, and since every step ends with bs_update the captured
        // step includes the rebuild of the tables that depend on the node positions
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        if (cudaStreamBeginCapture(ss, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const int rc2 = step(ss);
            const cudaError_t e2 = cudaStreamEndCapture(ss, &g);
            if (rc2 != BS_OK || e2 != cudaSuccess || !g || cudaGraphInstantiate(&x, g, 0) != cudaSuccess) x = nullptr;
        }
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();  // a capture that failed leaves no launch behind; the steps then run eagerly
        cudaError_t e = cudaSuccess;
        if (x) {
            for (; done < n_steps && e == cudaSuccess; ++done) e = cudaGraphLaunch(x, ss);
            h->graph_steps += done - 1;
            cudaGraphExecDestroy(x);
        }
        BS_CUDA(cudaEventRecord(h->step_out, ss));
        BS_CUDA(cudaStreamWaitEvent(caller, h->step_out, 0));
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    }
    for (; done < n_steps; ++done)
        if ((rc = step(stream))) return rc;
    return BS_OK;
}

int bs_graph_steps(bs_handle h, int64_t *steps)
{
    if (!h || !steps) return fail(BS_ERR_ARG, "NULL argument");
    *steps = h->graph_steps;
    return BS_OK;
}

namespace {

// near_walk (evaluation points = the mesh's nodes, hybrid rule): the mesh walk's arguments for the near field;
// used when the variant leaves the near pairs to a pass of their own.
int velocity_impl(bs_handle h, const double *eval_pts_dev, int64_t k, const bs_params *p, double *out_dev,
                  void *stream, const int *skip, const WalkArgs *near_walk)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    int rc = check_params(p);
    if (rc) return rc;
    if (k < 0) return fail(BS_ERR_ARG, "k < 0");
    if (k > INT32_MAX) return fail(BS_ERR_ARG, "k exceeds the int32 index range");
    if (k == 0) return BS_OK;
    if (!eval_pts_dev || !out_dev) return fail(BS_ERR_ARG, "NULL points or output");
    cudaStream_t st = (cudaStream_t)stream;
    if (h->n_tets == 0) {
        BS_CUDA(cudaMemsetAsync(out_dev, 0, sizeof(double) * 3 * k, st));
        if (p->counts) BS_CUDA(cudaMemsetAsync(p->counts, 0, sizeof(int32_t) * 3 * k, st));
        return BS_OK;
    }
    const int Q = p->tet_gauss_order;
    const int L = p->n_phi * p->n_theta;
    BS_CUDA(ensure_lines(h, p->n_phi, p->n_theta, st));
    // far_ratio = +inf: every pair takes the ray rule, in the all-ray kernel (one point per thread,
    // direction windows, the direction table in shared memory: up to kRayLinesSmemMax lines);
    // BS_ALLRAY_GENERIC=1 keeps such calls on the velocity kernel
    const char *generic_env = getenv("BS_ALLRAY_GENERIC");
    const bool ray = isinf(p->far_ratio) && L <= kRayLinesSmemMax && !(generic_env && atoi(generic_env) != 0) &&
                     p->near_rule == BS_NEAR_RAY;
    const int variant = ray ? 0 : choose_variant(h, p, k, near_walk != nullptr);
    const LaunchShape shape = ray ? ray_shape() : shape_for(p->precision, Q, variant, p->near_rule);
    if (!ray) BS_CUDA(ensure_far(h, Q, shape.tile, shape.layout, st));
    int occ_ray = 0;
    if (ray) {
        if (h->ray_occ[p->precision] == 0 || h->ray_occ_L[p->precision] != L) {
            h->ray_occ[p->precision] = std::max(1, ray_ctas_per_sm(p->precision, L));
            h->ray_occ_L[p->precision] = L;
        }
        occ_ray = h->ray_occ[p->precision];
    }
    int &occ = ray ? occ_ray : h->occ[p->near_rule][p->precision][Q][variant];
    if (occ == 0) occ = std::max(1, velocity_ctas_per_sm(p->precision, Q, variant, p->near_rule));
    const int64_t BP = (int64_t)shape.threads * shape.points_per_thread;
    const int64_t n_blocks = (k + BP - 1) / BP;
    const int64_t n_tiles = (h->n_tets + shape.tile - 1) / shape.tile;
    const int64_t slots = (int64_t)h->n_sm * occ;
    const int64_t target = 16LL * slots;
    const int64_t c0 = std::min<int64_t>(std::max<int64_t>((target + n_blocks - 1) / n_blocks, 1), n_tiles);
    // at least kMinTilesPerItem tiles per item (shorter items are dominated by their set-up), unless that
    // leaves the GPU with fewer items than it has CTA slots
    const int64_t min_per =
        n_blocks * ((n_tiles + kMinTilesPerItem - 1) / kMinTilesPerItem) < slots ? 1 : kMinTilesPerItem;
    // the persistent CTAs pull equal items, so the launch takes about ceil(items / slots) item times: of the chunk
    // counts c0..2 c0, take the one with the least waves x tiles per item (the last wave as full as it can be)
    int64_t per = 0, n_chunks = 0, best = 0;
    for (int64_t c = c0; c <= std::min<int64_t>({2 * c0, c0 + 256, n_tiles}); ++c) {
        const int64_t pc = std::min<int64_t>(std::max<int64_t>((n_tiles + c - 1) / c, min_per), n_tiles);
        const int64_t cc = (n_tiles + pc - 1) / pc;
        const int64_t cost = ((n_blocks * cc + slots - 1) / slots) * pc;
        if (n_chunks == 0 || cost < best) {
            best = cost;
            per = pc;
            n_chunks = cc;
        }
    }

    const int bits = order_grid_bits(k);
    BS_CUDA(ensure_order(h, k, bits, st));
    BS_CUDA(ensure_partial(h, sizeof(double) * 3 * (size_t)k * n_chunks, st));
    BS_CUDA(spatial_order(eval_pts_dev, k, bits, h->box, h->keys, h->cell_count, h->perm, st));

    VelocityArgs a;
    a.m.n_tets = h->n_tets;
    a.m.far = p->precision == BS_FP32 ? (const void *)h->far32 : (const void *)h->far64;
    a.m.near32 = h->near32;
    a.m.near64 = h->near64;
    a.m.tile_hdr = h->tile_hdr;
    a.m.pts = eval_pts_dev;
    a.m.perm = h->perm;
    a.m.k = k;
    a.Q = Q;
    set_far_ratio(a, p->far_ratio);
    a.lines = h->lines;
    a.L = L;
    a.smem_lines = a.L <= (ray ? kRayLinesSmemMax : kSmemLinesMax) ? 1 : 0;
    a.counts = p->counts;
    a.m.out = out_dev;
    a.flag = h->flag;
    a.work_counter = h->work_counter;
    a.m.n_chunks = (int)n_chunks;
    a.m.tiles_per_chunk = (int)per;
    a.m.partial = h->partial;
    a.variant = variant;
    a.skip = skip;
    a.near_rule = p->near_rule;
    a.n_items = n_blocks * n_chunks;
    if (a.n_items > INT32_MAX) return fail(BS_ERR_ARG, "too many work items for one launch (points x tet chunks)");
    a.wait_polls = h->copy_wait_polls;
    a.withhold_copies = h->withhold_copies;
    if (!ray && shape.drain == 3) {  // the near pass evaluates the near pairs the far sweep leaves out
        // without the walk, few points split the tiles among several CTAs per group of 32 points (each part at
        // least one group of 32 tiles per warp), for about kNearPassBlocksPerSm CTAs per SM in all
        const int64_t groups = (k + 31) / 32;
        const int64_t tile_groups = (h->n_tets + 32LL * shape.tile - 1) / (32LL * shape.tile);
        int64_t split = 1;
        if (!near_walk) {
            const int64_t want = ((int64_t)kNearPassBlocksPerSm * h->n_sm + groups - 1) / groups;
            split = std::max<int64_t>(1, std::min<int64_t>({want, tile_groups / kNearPassWarps, 16}));
        }
        const size_t need = 3 * (size_t)k * (size_t)split;
        if (need > h->near_cap) {
            if (h->near_out) cudaFreeAsync(h->near_out, st);
            h->near_out = nullptr;
            h->near_cap = 0;
            BS_CUDA(cudaMallocAsync((void **)&h->near_out, sizeof(double) * need, st));
            h->near_cap = need;
        }
        a.near_out = h->near_out;
        a.tile = shape.tile;
        a.far_stride = p->precision == BS_FP32 ? far_stride<float>(Q, shape.layout) : far_stride<double>(Q);
        a.n_near_warps = groups;
        a.near_split = (int)split;
        a.near_split_stride = 3 * k;
    }
    int grid = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->prof) {
        if (h->ev_free.empty()) {
            BS_CUDA(cudaEventCreate(&e0));
            BS_CUDA(cudaEventCreate(&e1));
        } else {
            e0 = h->ev_free.back().first;
            e1 = h->ev_free.back().second;
            h->ev_free.pop_back();
        }
        h->ev_used.push_back({e0, e1});
    }
    int extra = 0;  // kernels launched beyond zero, velocity and reduce (for bs_profile)
    if (ray) {
        BS_CUDA(launch_ray(p->precision, a, h->n_sm, st, &grid, e0, e1));
    } else {
        BS_CUDA(launch_velocity(p->precision, a, h->n_sm, st, &grid, e0, nullptr));
        if (shape.drain == 3) {  // the near field: by the mesh walk at the nodes when it can, else the near pass
            if (near_walk) {
                WalkArgs w = *near_walk;
                w.perm = h->perm;
                w.near_out = a.near_out;
                w.far = a.m.far;
                w.tile_hdr = h->tile_hdr;
                w.tile = a.tile;
                w.far_stride = a.far_stride;
                w.far_ratio2_f = a.far_ratio2_f;
                w.far_ratio2 = a.far_ratio2;
                w.counts = p->counts;
                BS_CUDA(launch_walk(p->precision, w, st));
                a.near_skip = near_walk->mode;  // the walk is in charge unless the mesh is not conforming
                extra += 2;
            }
            BS_CUDA(launch_near_pass(p->precision, a, st));
            extra += 1;
        }
        if (e1) BS_CUDA(cudaEventRecord(e1, st));
    }
    BS_CUDA(launch_reduce(a, st));
    if (h->prof) {
        h->prof_kernel += 1;
        h->prof_all += 5 /* ordering */ + 3 /* zero, velocity, reduce */ + extra;
    }
    return BS_OK;
}

// The batch's near walks, one per mesh, spread over side streams so that several meshes' walks share the GPU (a
// small mesh's walk is about one wave of warps whose gathers wait on one another) and overlap the far kernel, which
// they do not depend on (they read the meshes' tables and write their own meshes' near totals).  fork_batch_walks:
// the side streams wait on an event recorded on st, take the walks largest mesh first in turn, and each records
// its join event; join_batch_walks: st waits on those.  Their order does not change the result.  Inside a stream
// capture this records the walks as parallel branches of the graph.  Every side stream that waited on the fork
// records its join event, whatever fails in between, and *forked marks it, so that a capture can always end.
cudaError_t ensure_walk_streams(bs_batch_ctx *b)
{
    while ((int)b->walk_streams.size() < kBatchWalkStreams) {
        cudaStream_t s = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        b->walk_streams.push_back(s);
    }
    while ((int)b->walk_events.size() < kBatchWalkStreams + 1) {
        cudaEvent_t e = nullptr;
        cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (r != cudaSuccess) return r;
        b->walk_events.push_back(e);
    }
    return cudaSuccess;
}

cudaError_t fork_batch_walks(bs_batch_ctx *b, int prec, cudaStream_t st, unsigned *forked)
{
    *forked = 0;
    const int n = (int)b->walks.size();
    if (n == 0) return cudaSuccess;
    if ((int)b->walk_streams.size() < kBatchWalkStreams || (int)b->walk_events.size() < kBatchWalkStreams + 1)
        return cudaErrorNotReady;  // ensure_walk_streams was not called (it runs outside any capture)
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->walks[x].n_nodes > b->walks[y].n_nodes; });
    const int K = std::min(n, (int)b->walk_streams.size());
    cudaError_t first = cudaEventRecord(b->walk_events[0], st);
    if (first != cudaSuccess) return first;
    for (int k = 0; k < K; ++k) {
        cudaStream_t s = b->walk_streams[k];
        cudaError_t e = cudaStreamWaitEvent(s, b->walk_events[0], 0);
        if (e != cudaSuccess) {  // not forked: nothing to join
            if (first == cudaSuccess) first = e;
            continue;
        }
        for (int i = k; first == cudaSuccess && i < n; i += K) {
            e = launch_walk(prec, b->walks[order[i]], s);
            if (e != cudaSuccess) first = e;
        }
        e = cudaEventRecord(b->walk_events[1 + k], s);
        if (e == cudaSuccess)
            *forked |= 1u << k;
        else if (first == cudaSuccess)
            first = e;
    }
    return first;
}

cudaError_t join_batch_walks(bs_batch_ctx *b, cudaStream_t st, unsigned forked)
{
    cudaError_t first = cudaSuccess;
    for (int k = 0; k < (int)b->walk_streams.size(); ++k)
        if (forked & (1u << k)) {
            const cudaError_t e = cudaStreamWaitEvent(st, b->walk_events[1 + k], 0);
            if (e != cudaSuccess && first == cudaSuccess) first = e;
        }
    return first;
}

}  // namespace

int bs_velocity_host(bs_handle h, const double *eval_pts_host, int64_t k, const bs_params *p, double *out_host,
                     void *stream)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    int rc = check_params(p);
    if (rc) return rc;
    if (k < 0) return fail(BS_ERR_ARG, "k < 0");
    if (k == 0) return BS_OK;
    if (!eval_pts_host || !out_host) return fail(BS_ERR_ARG, "NULL points or output");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * 3 * (size_t)k;
    if (2 * bytes > h->stage_cap) {
        if (h->stage) cudaFreeAsync(h->stage, st);
        h->stage = nullptr;
        h->stage_cap = 0;
        BS_CUDA(cudaMallocAsync((void **)&h->stage, 2 * bytes, st));
        h->stage_cap = 2 * bytes;
    }
    double *dpts = h->stage, *dout = h->stage + 3 * k;
    BS_CUDA(cudaMemcpyAsync(dpts, eval_pts_host, bytes, cudaMemcpyHostToDevice, st));
    rc = bs_velocity(h, dpts, k, p, dout, stream);
    if (rc) return rc;
    BS_CUDA(cudaMemcpyAsync(out_host, dout, bytes, cudaMemcpyDeviceToHost, st));
    BS_CUDA(cudaStreamSynchronize(st));
    return BS_OK;
}

int bs_destroy(bs_handle h)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    cudaDeviceSynchronize();
    free_ctx(h);
    return BS_OK;
}

int bs_direction_table(int n_phi, int n_theta, double *s_host, double *k_host)
{
    if (n_phi < 1 || n_phi > 256 || n_theta < 1 || n_theta > 256) return fail(BS_ERR_ARG, "n_phi/n_theta out of 1..256");
    if (!s_host || !k_host) return fail(BS_ERR_ARG, "NULL output");
    const size_t L = (size_t)n_phi * n_theta;
    float4 *f = nullptr;
    dbl4 *d = nullptr;
    BS_CUDA(cudaMalloc(&f, L * sizeof(float4)));
    cudaError_t e = cudaMalloc(&d, L * sizeof(dbl4));
    if (e == cudaSuccess) e = build_lines(n_phi, n_theta, f, d, 0);
    dbl4 *hd = new dbl4[L];
    if (e == cudaSuccess) e = cudaMemcpy(hd, d, L * sizeof(dbl4), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        for (size_t l = 0; l < L; ++l) {
            s_host[3 * l] = hd[l].x;
            s_host[3 * l + 1] = hd[l].y;
            s_host[3 * l + 2] = hd[l].z;
            k_host[l] = hd[l].w;
        }
    delete[] hd;
    cudaFree(f);
    if (d) cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "bs_direction_table");
    return BS_OK;
}

int bs_tet_rule(int order, double *bary_host, double *w_host)
{
    if (!valid_order(order)) return fail(BS_ERR_ORDER, "tet_gauss_order must be 1, 4, 8, 27 or 64");
    if (!bary_host || !w_host) return fail(BS_ERR_ARG, "NULL output");
    double *b = nullptr, *w = nullptr;
    BS_CUDA(cudaMalloc(&b, sizeof(double) * 4 * order));
    cudaError_t e = cudaMalloc(&w, sizeof(double) * order);
    if (e == cudaSuccess) e = build_tet_rule(order, b, w, 0);
    if (e == cudaSuccess) e = cudaMemcpy(bary_host, b, sizeof(double) * 4 * order, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(w_host, w, sizeof(double) * order, cudaMemcpyDeviceToHost);
    cudaFree(b);
    if (w) cudaFree(w);
    if (e != cudaSuccess) return cuda_fail(e, "bs_tet_rule");
    return BS_OK;
}

int bs_profile(bs_handle h, int enable)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    h->prof = enable != 0;
    drop_events(h);
    h->prof_kernel = h->prof_all = 0;
    return BS_OK;
}

int bs_profile_read(bs_handle h, double *kernel_ms, int64_t *kernel_launches, int64_t *all_launches)
{
    if (!h || !kernel_ms || !kernel_launches || !all_launches) return fail(BS_ERR_ARG, "NULL argument");
    BS_CUDA(cudaDeviceSynchronize());
    double total = 0.0;
    for (auto &p : h->ev_used) {
        float ms = 0.f;
        BS_CUDA(cudaEventElapsedTime(&ms, p.first, p.second));
        total += ms;
    }
    *kernel_ms = total;
    *kernel_launches = h->prof_kernel;
    *all_launches = h->prof_all;
    return BS_OK;
}

int bs_batch_create(const bs_handle *meshes, int n, bs_batch *out)
{
    if (!out) return fail(BS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!meshes || n < 1) return fail(BS_ERR_ARG, "need at least one mesh");
    for (int i = 0; i < n; ++i)
        if (!meshes[i]) return fail(BS_ERR_ARG, "NULL mesh handle in the batch");
    bs_batch_ctx *b = new bs_batch_ctx();
    b->meshes.assign(meshes, meshes + n);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        b->point_begin.push_back(total);
        total += meshes[i]->n_nodes;
    }
    b->n_points = total;
    b->order_version.assign(n, 0);
    if (e == cudaSuccess) e = cudaMalloc(&b->perm, sizeof(int) * total);
    if (e == cudaSuccess) e = cudaMalloc(&b->keys, sizeof(unsigned) * total);
    if (e == cudaSuccess) e = cudaMalloc(&b->box, sizeof(int) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_meshes, sizeof(MeshDesc) * n);
    if (e == cudaSuccess) e = cudaMalloc(&b->work_counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&b->flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->flag, 0, sizeof(int));
    int64_t kmax = 1;
    for (int i = 0; i < n; ++i) kmax = std::max(kmax, meshes[i]->n_nodes);
    b->cell_bits = order_grid_bits(kmax);
    if (e == cudaSuccess) e = cudaMalloc(&b->cell_count, sizeof(int) << (3 * b->cell_bits));
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "bs_batch_create");
    }
    *out = b;
    return BS_OK;
}

int bs_batch_velocity(bs_batch b, const bs_params *p, double *const *outs, void *stream)
{
    if (!b) return fail(BS_ERR_ARG, "batch is NULL");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->counts) return fail(BS_ERR_ARG, "bs_batch_velocity: counts are not supported (set p->counts = NULL)");
    if (!outs) return fail(BS_ERR_ARG, "outs is NULL");
    const int n = (int)b->meshes.size();
    for (int i = 0; i < n; ++i)
        if (!outs[i]) return fail(BS_ERR_ARG, "NULL output in outs");
    cudaStream_t st = (cudaStream_t)stream;
    const int Q = p->tet_gauss_order;
    const int prec = p->precision;
    bool changed = false;

    // the variant: BS_VARIANT, else the first mesh's pinned variant (bs_set_variant), else (ray rule) variant 0
    // when it leaves the near pairs to the near pass, else the one-point-per-thread variant for batches of small
    // meshes, else variant 0
    const int nr = p->near_rule;
    const int nv = num_variants(prec, Q, nr);
    int variant = b->meshes[0]->pinned[nr][prec][Q];
    const char *variant_env = getenv("BS_VARIANT");
    if (variant_env) variant = atoi(variant_env);
    if (variant < 0 || variant >= nv) {
        variant = 0;
        if (!variant_env && nr == BS_NEAR_RAY) {
            int64_t largest = 0;
            for (int i = 0; i < n; ++i) largest = std::max(largest, b->meshes[i]->n_tets);
            const int sv = small_mesh_variant(prec, Q, false);
            // a variant that leaves the near pairs to the near pass, which then covers every mesh's points in
            // one launch; else, for small meshes, one point per thread with the pairs drained in the kernel
            if (shape_for(prec, Q, 0, nr).drain == 3) variant = 0;
            else if (sv >= 0 && largest <= kSmallBatchMeshTets) variant = sv;
        }
    }
    const LaunchShape shape = shape_for(prec, Q, variant, nr);

    // per-mesh tables (rebuilt only when stale) and per-mesh point orders (nodes = evaluation points)
    for (int i = 0; i < n; ++i) {
        bs_ctx *h = b->meshes[i];
        const uint64_t before = h->far_version;
        const int before_q = h->rule.order, before_tile = h->far_tile, before_layout = h->far_layout;
        BS_CUDA(ensure_far(h, Q, shape.tile, shape.layout, st));
        changed = changed || before != h->far_version || before_q != h->rule.order || before_tile != h->far_tile ||
                  before_layout != h->far_layout;
        if (b->order_version[i] != h->version) {
            const int bits = order_grid_bits(h->n_nodes);
            BS_CUDA(spatial_order(h->nodes, h->n_nodes, bits, b->box, b->keys, b->cell_count,
                                  b->perm + b->point_begin[i], st));
            b->order_version[i] = h->version;
        }
    }
    if (!b->lines.f32 || b->lines.n_phi != p->n_phi || b->lines.n_theta != p->n_theta) {
        if (b->lines.f32) cudaFreeAsync(b->lines.f32, st);
        if (b->lines.f64) cudaFreeAsync(b->lines.f64, st);
        b->lines = LineTables();
        const size_t L = (size_t)p->n_phi * p->n_theta;
        BS_CUDA(cudaMallocAsync((void **)&b->lines.f32, L * sizeof(float4), st));
        BS_CUDA(cudaMallocAsync((void **)&b->lines.f64, L * sizeof(dbl4), st));
        BS_CUDA(build_lines(p->n_phi, p->n_theta, b->lines.f32, b->lines.f64, st));
        b->lines.n_phi = p->n_phi;
        b->lines.n_theta = p->n_theta;
        changed = true;
    }

    // decomposition: items of roughly equal work over all meshes
    int &occ = b->meshes[0]->occ[nr][prec][Q][variant];
    if (occ == 0) occ = std::max(1, velocity_ctas_per_sm(prec, Q, variant, p->near_rule));
    const int64_t BP = (int64_t)shape.threads * shape.points_per_thread;
    double total_pairs = 0.0;
    for (int i = 0; i < n; ++i) total_pairs += (double)b->meshes[i]->n_nodes * b->meshes[i]->n_tets;
    const double per_item = std::max(1.0, total_pairs / (16.0 * b->n_sm * occ));
    std::vector<MeshDesc> md(n);
    int64_t items = 0, partial_elems = 0, near_warps = 0;
    for (int i = 0; i < n; ++i) {
        bs_ctx *h = b->meshes[i];
        MeshDesc &m = md[i];
        m.near_warp_begin = near_warps;
        near_warps += (h->n_nodes + 31) / 32;
        const int64_t k = h->n_nodes;
        const int64_t n_tiles = std::max<int64_t>(1, (h->n_tets + shape.tile - 1) / shape.tile);
        const double block_pairs = (double)std::min<int64_t>(BP, k) * shape.tile;
        int64_t per = (int64_t)std::ceil(per_item / block_pairs);
        per = std::min<int64_t>(std::max<int64_t>(per, kMinTilesPerItem), n_tiles);
        // a mesh without tets owns no items and no partial sums: the reduction writes zeros
        const int64_t n_chunks = h->n_tets > 0 ? (n_tiles + per - 1) / per : 0;
        m.far = prec == BS_FP32 ? (const void *)h->far32 : (const void *)h->far64;
        m.near32 = h->near32;
        m.near64 = h->near64;
        m.tile_hdr = h->tile_hdr;
        m.pts = h->nodes;
        m.perm = b->perm + b->point_begin[i];
        m.out = outs[i];
        m.k = k;
        m.n_tets = h->n_tets;
        m.n_chunks = (int)n_chunks;
        m.tiles_per_chunk = (int)per;
        m.item_begin = items;
        m.point_begin = b->point_begin[i];
        items += h->n_tets > 0 ? ((k + BP - 1) / BP) * n_chunks : 0;
        m.partial = reinterpret_cast<double *>(partial_elems);  // offset, fixed below
        partial_elems += 3 * k * n_chunks;
    }
    if ((size_t)partial_elems * sizeof(double) > b->partial_cap) {
        if (b->partial) cudaFreeAsync(b->partial, st);
        b->partial = nullptr;
        b->partial_cap = 0;
        BS_CUDA(cudaMallocAsync((void **)&b->partial, sizeof(double) * partial_elems, st));
        b->partial_cap = sizeof(double) * partial_elems;
        changed = true;
    }
    for (int i = 0; i < n; ++i) md[i].partial = b->partial + reinterpret_cast<intptr_t>(md[i].partial);
    if (shape.drain == 3 && !b->near_out) {  // the near pass's totals, all meshes' points
        BS_CUDA(cudaMallocAsync((void **)&b->near_out, sizeof(double) * 3 * std::max<int64_t>(b->n_points, 1), st));
        changed = true;
    }
    // The near field of a variant that leaves it out: at the meshes' nodes, the mesh walk of each mesh (its tables
    // prepared here, outside any capture) where the mesh allows it; the near pass skips those meshes.
    const int L = p->n_phi * p->n_theta;
    const char *walk_env = getenv("BS_WALK");
    const bool batch_walk = shape.drain == 3 && nr == BS_NEAR_RAY && L <= kRayLinesSmemMax &&
                            !(walk_env && atoi(walk_env) == 0);
    std::vector<WalkArgs> walks;
    if (batch_walk) {
        double fr2 = 0.0;
        float fr2f = 0.f;
        {
            VelocityArgs t;
            set_far_ratio(t, p->far_ratio);
            fr2 = t.far_ratio2;
            fr2f = t.far_ratio2_f;
        }
        for (int i = 0; i < n; ++i) {
            bs_ctx *h = b->meshes[i];
            if (h->n_tets == 0) continue;
            BS_CUDA(walk_prepare(h, st));
            BS_CUDA(ensure_rstop(h, p->far_ratio, st));
            WalkArgs w;
            std::memset(static_cast<void *>(&w), 0, sizeof(w));  // padding too: compared byte for byte
            walk_args(h, w);
            w.lines32 = b->lines.f32;
            w.lines64 = b->lines.f64;
            w.L = L;
            w.out = outs[i];
            w.near_mode = 1;
            w.perm = md[i].perm;
            w.near_out = b->near_out + 3 * md[i].point_begin;
            w.far = md[i].far;
            w.tile_hdr = h->tile_hdr;
            w.tile = shape.tile;
            w.far_stride = prec == BS_FP32 ? far_stride<float>(Q, shape.layout) : far_stride<double>(Q);
            w.far_ratio2_f = fr2f;
            w.far_ratio2 = fr2;
            w.r_stop = h->r_stop;
            walks.push_back(w);
        }
    }
    // per mesh, the flag the near pass reads to leave a walked mesh alone (the walk's mode: set when it is in charge)
    std::vector<const int *> skips(n, nullptr);
    if (batch_walk)
        for (int i = 0; i < n; ++i)
            if (b->meshes[i]->n_tets > 0) skips[i] = b->meshes[i]->walk_mode;
    if (batch_walk && !b->d_near_skip) {
        BS_CUDA(cudaMallocAsync((void **)&b->d_near_skip, sizeof(int *) * n, st));
        changed = true;
    }
    if (batch_walk && skips != b->h_near_skip) {
        BS_CUDA(cudaMemcpyAsync(b->d_near_skip, skips.data(), sizeof(int *) * n, cudaMemcpyHostToDevice, st));
        BS_CUDA(cudaStreamSynchronize(st));  // skips is a host temporary
        b->h_near_skip = skips;
        changed = true;
    }
    if (!walks.empty()) BS_CUDA(ensure_walk_streams(b));
    if (walks.size() != b->walks.size() ||
        (!walks.empty() && memcmp(walks.data(), b->walks.data(), sizeof(WalkArgs) * walks.size()) != 0)) {
        b->walks = walks;
        changed = true;
    }

    const bool same_desc = b->h_meshes.size() == md.size() &&
                           memcmp(b->h_meshes.data(), md.data(), sizeof(MeshDesc) * md.size()) == 0;
    if (!same_desc) {
        BS_CUDA(cudaMemcpyAsync(b->d_meshes, md.data(), sizeof(MeshDesc) * n, cudaMemcpyHostToDevice, st));
        BS_CUDA(cudaStreamSynchronize(st));  // md is a host temporary
        b->h_meshes = md;
        changed = true;
    }

    VelocityArgs a;
    std::memset(static_cast<void *>(&a), 0, sizeof(a));  // padding too: the graph cache compares bytes
    a.meshes = b->d_meshes;
    a.n_meshes = n;
    a.n_items = items;
    if (items > INT32_MAX) return fail(BS_ERR_ARG, "too many work items for one batch launch");
    a.n_points = b->n_points;
    a.Q = Q;
    set_far_ratio(a, p->far_ratio);
    a.lines = b->lines;
    a.L = p->n_phi * p->n_theta;
    a.smem_lines = a.L <= kSmemLinesMax ? 1 : 0;
    a.flag = b->flag;
    a.work_counter = b->work_counter;
    a.variant = variant;
    a.near_rule = p->near_rule;
    a.wait_polls = b->meshes[0]->copy_wait_polls;  // the batch follows its first mesh's wait limits
    a.withhold_copies = b->meshes[0]->withhold_copies;
    if (shape.drain == 3) {
        a.near_out = b->near_out;
        a.tile = shape.tile;
        a.far_stride = prec == BS_FP32 ? far_stride<float>(Q, shape.layout) : far_stride<double>(Q);
        a.n_near_warps = near_warps;
        if (batch_walk) a.mesh_near_skip = b->d_near_skip;
    }
    if (items == 0) {  // every mesh is empty: the reduction alone writes the zeros
        BS_CUDA(launch_reduce(a, st));
        return BS_OK;
    }

    // the launch sequence {zero counter, persistent velocity kernel, near walks, near pass, batched reduction} is
    // captured
    // once per (launch arguments, stream) into a CUDA graph and replayed
    const bool graphable = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
    const bool same_graph = b->graph && !changed && b->graph_stream == st && b->graph_prec == prec &&
                            memcmp(&b->graph_args, &a, sizeof(a)) == 0;
    if (graphable && !same_graph) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        // attributes and occupancy are set outside the capture
        BS_CUDA(velocity_ctas_per_sm(prec, Q, variant, nr) > 0 ? cudaSuccess : cudaErrorUnknown);
        cudaGraph_t g = nullptr;
        BS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int grid = 0;
        unsigned forked = 0;
        cudaError_t e1 = fork_batch_walks(b, prec, st, &forked);
        if (e1 == cudaSuccess) e1 = launch_velocity(prec, a, b->n_sm, st, &grid);
        const cudaError_t ej = join_batch_walks(b, st, forked);
        if (e1 == cudaSuccess) e1 = ej;
        if (e1 == cudaSuccess) e1 = launch_near_pass(prec, a, st);  // no-op unless the variant leaves near pairs
        cudaError_t e2 = e1 == cudaSuccess ? launch_reduce(a, st) : e1;
        cudaError_t e3 = cudaStreamEndCapture(st, &g);
        if (e2 != cudaSuccess) return cuda_fail(e2, "bs_batch_velocity (capture)");
        if (e3 != cudaSuccess) return cuda_fail(e3, "cudaStreamEndCapture");
        cudaError_t e4 = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e4 != cudaSuccess) return cuda_fail(e4, "cudaGraphInstantiate");
        b->graph_stream = st;
        b->graph_prec = prec;
        b->graph_args = a;
    }
    if (graphable) {
        BS_CUDA(cudaGraphLaunch(b->graph, st));
    } else {
        int grid = 0;
        unsigned forked = 0;
        cudaError_t e1 = fork_batch_walks(b, prec, st, &forked);
        if (e1 == cudaSuccess) e1 = launch_velocity(prec, a, b->n_sm, st, &grid);
        const cudaError_t ej = join_batch_walks(b, st, forked);
        BS_CUDA(e1);
        BS_CUDA(ej);
        BS_CUDA(launch_near_pass(prec, a, st));
        BS_CUDA(launch_reduce(a, st));
    }
    return BS_OK;
}

int bs_batch_status(bs_batch b, void *stream)
{
    if (!b) return fail(BS_ERR_ARG, "batch is NULL");
    BS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int flag = 0;
    BS_CUDA(cudaMemcpy(&flag, b->flag, sizeof(int), cudaMemcpyDeviceToHost));
    BS_CUDA(cudaMemset(b->flag, 0, sizeof(int)));
    // the meshes' own flags: their tables (bs_update) and their near walks
    int rc = BS_OK;
    for (bs_ctx *h : b->meshes) {
        const int r = bs_status(h, stream);
        if (r != BS_OK && rc == BS_OK) rc = r;
    }
    if (flag & kFlagTimeout) return fail(BS_ERR_TIMEOUT, "a bounded device wait of the batch gave up");
    if (flag & (kFlagMeshIndex | kFlagMeshVolume)) return fail(BS_ERR_MESH, "degenerate tet in the batch");
    return rc;
}

int bs_batch_destroy(bs_batch b)
{
    if (!b) return fail(BS_ERR_ARG, "batch is NULL");
    cudaDeviceSynchronize();
    free_batch(b);
    return BS_OK;
}

}  // extern "C"

namespace {

// bs_autotune for one path: the points path (bs_velocity at the mesh's nodes: arbitrary points) or the nodes
// path (bs_velocity_nodes, where the mesh walk can take the near field).  A cache hit takes the stored
// variant; else every variant is pinned in turn and timed.  *chosen: the variant.
int tune_path(bs_handle h, const bs_params *p, void *stream, bool at_nodes, int *chosen)
{
    cudaStream_t st = (cudaStream_t)stream;
    const int prec = p->precision, Q = p->tet_gauss_order, nr = p->near_rule;
    const int L = p->n_phi * p->n_theta;
    const int nv = num_variants(prec, Q, nr);
    const int64_t k = h->n_nodes;
    const std::string key = tune_key(h->gpu_name, h->n_sm, prec, Q, nr, L, k, h->n_tets, at_nodes);
    const char *force = getenv("BS_TUNE_FORCE");
    if (!(force && atoi(force) != 0)) {
        const int v = tune_lookup(key, prec, Q, nr);
        if (v >= 0 && v < nv) {  // a cache hit: no timing
            h->tune_memo[key] = v;
            *chosen = v;
            return BS_OK;
        }
    }
    double *out = nullptr;
    BS_CUDA(cudaMallocAsync((void **)&out, sizeof(double) * 3 * h->n_nodes, st));
    bs_params q = *p;
    q.counts = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = INFINITY;
    int best_v = 0, rc = BS_OK;
    const int saved = h->pinned[nr][prec][Q];
    auto call = [&]() {
        return at_nodes ? bs_velocity_nodes(h, &q, out, stream) : bs_velocity(h, h->nodes, k, &q, out, stream);
    };
    for (int v = 0; v < nv && e == cudaSuccess && rc == BS_OK; ++v) {
        h->pinned[nr][prec][Q] = v;
        rc = call();  // warm-up (also builds this variant's tables)
        double total = 0.0;
        int reps = 0;
        // at least one timed call, more while they take under 20 ms in all (at most 10)
        while (rc == BS_OK && e == cudaSuccess && reps < 10 && (reps == 0 || total < 20.0)) {
            if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
            rc = call();
            if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.f;
            if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
            total += ms;
            ++reps;
        }
        if (reps > 0 && total / reps < best) {
            best = total / reps;
            best_v = v;
        }
    }
    h->pinned[nr][prec][Q] = saved;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    if (e != cudaSuccess) return cuda_fail(e, "bs_autotune");
    if (rc) return rc;
    BS_CUDA(cudaStreamSynchronize(st));
    if (int fs = bs_status(h, stream)) return fs;  // a timed call raised the flag: keep nothing
    h->tune_memo[key] = best_v;
    *chosen = best_v;
    // persisted where the cache file is writable; kept for this process in any case
    tune_store(key, prec, Q, nr, best_v, best, nv);
    return BS_OK;
}

}  // namespace

extern "C" {

int bs_autotune(bs_handle h, const bs_params *p, void *stream)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    int rc = check_params(p);
    if (rc) return rc;
    const int prec = p->precision, Q = p->tet_gauss_order, nr = p->near_rule;
    const int L = p->n_phi * p->n_theta;
    h->tuned[0][nr][prec][Q] = h->tuned[1][nr][prec][Q] = 0;
    // nothing to choose: no tets, or the calls would run the all-ray kernel or the all-ray walk (one shape)
    const char *generic_env = getenv("BS_ALLRAY_GENERIC");
    const bool ray = isinf(p->far_ratio) && L <= kRayLinesSmemMax && !(generic_env && atoi(generic_env) != 0) &&
                     nr == BS_NEAR_RAY;
    if (h->n_tets == 0 || ray || num_variants(prec, Q, nr) <= 0) return BS_OK;
    int v = 0;
    if ((rc = tune_path(h, p, stream, false, &v))) return rc;
    h->tuned[0][nr][prec][Q] = v;
    // the nodes path differs where the mesh walk can take the near field (the hybrid rule, the ray near rule)
    const char *env = getenv("BS_WALK");
    if (!isinf(p->far_ratio) && L <= kRayLinesSmemMax && nr == BS_NEAR_RAY && !(env && atoi(env) == 0)) {
        if ((rc = tune_path(h, p, stream, true, &v))) return rc;
    }
    h->tuned[1][nr][prec][Q] = v;
    return BS_OK;
}

int bs_tuned_variant(bs_handle h, int precision, int tet_gauss_order, int at_nodes, int *variant)
{
    if (!h || !variant || (precision != BS_FP32 && precision != BS_FP64) || !valid_order(tet_gauss_order) ||
        (at_nodes != 0 && at_nodes != 1))
        return fail(BS_ERR_ARG, "bad argument");
    *variant = h->tuned[at_nodes][BS_NEAR_RAY][precision][tet_gauss_order];
    return BS_OK;
}

int bs_num_variants(int precision, int tet_gauss_order, int near_rule, int *n)
{
    if (!n || (precision != BS_FP32 && precision != BS_FP64) || (near_rule != BS_NEAR_RAY && near_rule != BS_NEAR_EXACT))
        return fail(BS_ERR_ARG, "bad argument");
    if (!valid_order(tet_gauss_order)) return fail(BS_ERR_ORDER, "tet_gauss_order must be 1, 4, 8, 27 or 64");
    *n = num_variants(precision, tet_gauss_order, near_rule);
    return BS_OK;
}

int bs_variant_shape(int precision, int tet_gauss_order, int near_rule, int variant, int32_t *shape)
{
    int n = 0;
    int rc = bs_num_variants(precision, tet_gauss_order, near_rule, &n);
    if (rc) return rc;
    if (!shape || variant < 0 || variant >= n) return fail(BS_ERR_ARG, "variant out of range");
    const VariantShape &s = velocity_variants(precision, tet_gauss_order, near_rule).v[variant].s;
    const int32_t v[8] = {s.P, s.TILE, s.S, s.MINB, s.DR, s.U, s.PK ? 1 : 0, s.UJ};
    for (int i = 0; i < 8; ++i) shape[i] = v[i];
    return BS_OK;
}

int bs_set_variant(bs_handle h, int precision, int tet_gauss_order, int near_rule, int variant)
{
    if (!h) return fail(BS_ERR_ARG, "handle is NULL");
    int n = 0;
    int rc = bs_num_variants(precision, tet_gauss_order, near_rule, &n);
    if (rc) return rc;
    if (variant < -1 || variant >= n) return fail(BS_ERR_ARG, "variant out of range (-1 for automatic)");
    h->pinned[near_rule][precision][tet_gauss_order] = variant;
    return BS_OK;
}

}  // extern "C"
