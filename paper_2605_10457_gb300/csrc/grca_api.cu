// Host runtime of libgrca.so: the C ABI declared in include/grca.h.
//
// Owns the device scene buffer, the sensor tables, the per-ray scratch and
// the device work queues; builds the per-cast sensor descriptors; launches
// (or replays as a CUDA graph) the frame's kernel sequence; runs the
// launch-parameter autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "grca.h"
#include "grca_internal.h"

using namespace grca;

namespace {

constexpr int RING = 64;  // pinned staging slots for per-cast sensor descriptors

struct SensorHost {
    grca_sensor_desc d;
    std::vector<double> elev;
    std::vector<double> theta;   // per-ray azimuths (empty: uniform grid)
    bool full;
    uint32_t* d_mask = nullptr;  // device on/off bits (nullptr: every ray fires)
    double range_sigma = 0.0;
    uint64_t noise_seed = 0;
};

struct GraphKey {
    uint32_t n_sensors, n_rays, total_ch, flags, n_tris, tri_first, split_at;
    const void* out_dist;
    const void* out_tri;
    const void* tris;
    const void* keys;
    const void* dump;
    int cull_block, cull_bps, inline_max, chunk_rays;
    bool operator<(const GraphKey& o) const {
        return std::tie(n_sensors, n_rays, total_ch, flags, n_tris, tri_first, split_at, out_dist, out_tri, tris, keys,
                        dump, cull_block, cull_bps, inline_max, chunk_rays) <
               std::tie(o.n_sensors, o.n_rays, o.total_ch, o.flags, o.n_tris, o.tri_first, o.split_at, o.out_dist,
                        o.out_tri, o.tris, o.keys, o.dump, o.cull_block, o.cull_bps, o.inline_max, o.chunk_rays);
    }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

struct grca_ctx {
    int device = 0;
    // the last grca_cast_shard (its work buffers hold the queue that
    // grca_resolve_shard re-tests)
    bool shard_ready = false;
    CastArgs shard_args{};
    LaunchCfg shard_cfg;
    int n_sm = 152;
    grca_options opt{};
    LaunchCfg cfg;
    cudaStream_t cap_stream = nullptr;
    // host-to-device copies of dynamic vertices that overlap the elevation
    // cull of the static triangles (grca_cast_host)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_free = nullptr, ev_copied = nullptr;
    // asynchronous host casts: results go out on d2h_stream; ev_out holds, in
    // order, one event per cast whose copy-out may still be running
    static constexpr int OUT_RING = 8;
    cudaStream_t d2h_stream = nullptr;
    cudaEvent_t ev_decoded = nullptr;
    cudaEvent_t ev_out[OUT_RING] = {};
    uint32_t out_head = 0, out_count = 0;
    bool defer_bounds = false;  // prepare_cast leaves the group-box refresh to the caller

    float* d_tris = nullptr;
    float4* d_gb = nullptr;         // GACP-T_g boxes, one pair of float4 per 32-triangle group
    // static hierarchy of the hybrid pipeline over triangles [0, n_static)
    BvhNode* d_bvh_nodes = nullptr;
    uint32_t* d_bvh_prim = nullptr;
    float* d_bvh_tris = nullptr;
    uint32_t n_static = 0;
    bool bvh_stale = false;         // static triangles changed since the build
    double bvh_delta = 0.0;
    float bvh_lo[3] = {0, 0, 0}, bvh_hi[3] = {0, 0, 0};
    uint32_t pending_launches = 0;  // group-bound kernels launched since the last cast
    // triangles whose group boxes are stale: [gb_lo, gb_hi) (refreshed lazily,
    // by the first cast that runs the group cull)
    uint32_t gb_lo = 0, gb_hi = 0;
    uint32_t n_tris = 0;
    size_t tris_cap = 0;  // triangles

    std::vector<SensorHost> sensors;
    float2* d_ch = nullptr;
    double2* d_ch64 = nullptr;
    float2* d_ch_lo = nullptr;
    float2* d_az_lo = nullptr;
    float2* d_az = nullptr;
    double2* d_az64 = nullptr;
    uint16_t* d_lut = nullptr;
    std::vector<uint32_t> ch_off, az_off;
    std::vector<float> lut_lo, lut_inv_w;
    bool tables_dirty = true;

    unsigned long long* d_surv = nullptr;
    size_t surv_cap = 0;
    unsigned long long* d_keys = nullptr;
    unsigned long long* d_keys64 = nullptr;
    uint32_t* d_flag_bits = nullptr;
    uint32_t* d_flag_list = nullptr;
    size_t ray_cap = 0;

    BigPair* d_big = nullptr;
    PairSetup* d_setups = nullptr;
    uint4* d_chunks = nullptr;
    uint4* d_recheck = nullptr;
    uint32_t* d_qcount = nullptr;
    unsigned long long* d_counters = nullptr;
    uint32_t* d_error = nullptr;

    SensorDev* d_sens = nullptr;
    SensorDev* h_ring = nullptr;
    cudaEvent_t ring_ev[RING] = {};
    bool ring_used[RING] = {};
    int ring_pos = 0;

    float* d_out_dist = nullptr;
    uint32_t* d_out_tri = nullptr;
    size_t out_cap = 0;

    uint32_t* dump = nullptr;
    uint64_t dump_cap = 0;
    uint32_t* dump_count = nullptr;

    std::map<GraphKey, std::pair<cudaGraphExec_t, int>> graphs;  // graph, kernels it launches
    std::map<std::tuple<uint32_t, uint32_t, uint32_t, uint32_t>, LaunchCfg> tuned;

    uint64_t last_n_rays = 0;
    uint32_t last_launches = 0;
    std::string last_err;

    // per-kernel CUDA-event timing (grca_profile_*)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_next = 0;
    struct Pending {
        int kernel;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    cudaEvent_t open_ev[K_NUM];
    double total_ms[K_NUM] = {};
    uint64_t n_launch[K_NUM] = {};
};

static cudaEvent_t pool_event(grca_ctx* ctx) {
    if (ctx->ev_next == ctx->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->ev_pool.push_back(e);
    }
    return ctx->ev_pool[ctx->ev_next++];
}

static void drain_profile(grca_ctx* ctx) {
    for (auto& p : ctx->pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ctx->total_ms[p.kernel] += ms;
            ctx->n_launch[p.kernel] += 1;
        }
    }
    ctx->pending.clear();
    ctx->ev_next = 0;
}

static void profile_mark(void* user, int kernel, int phase, cudaStream_t st) {
    grca_ctx* ctx = (grca_ctx*)user;
    if (ctx->ev_next + 2 > 8192) drain_profile(ctx);
    cudaEvent_t e = pool_event(ctx);
    if (!e) return;
    cudaEventRecord(e, st);
    if (phase == 0) {
        ctx->open_ev[kernel] = e;
    } else {
        ctx->pending.push_back({kernel, ctx->open_ev[kernel], e});
    }
}

static grca_status cuda_fail(grca_ctx* c, cudaError_t e, const char* what) {
    if (c) c->last_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? GRCA_ERR_OOM : GRCA_ERR_CUDA;
}

#define CK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

static void free_graphs(grca_ctx* ctx) {
    for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second.first);
    ctx->graphs.clear();
}

namespace grca {
bool valid_axes(const double f[3], const double r[3], const double u[3]) {
    auto dot = [](const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
    const double* v[3] = {f, r, u};
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(v[i][k])) return false;
    for (int i = 0; i < 3; ++i) {
        if (std::fabs(dot(v[i], v[i]) - 1.0) > 1e-9) return false;
        for (int k = i + 1; k < 3; ++k)
            if (std::fabs(dot(v[i], v[k])) > 1e-9) return false;
    }
    return true;
}

// every condition grca_create_sensor places on a description, sizes included
bool sensor_desc_valid(const grca_sensor_desc* d) {
    if (!d || !d->elev_rad) return false;
    if (d->n_channels < 1 || d->n_channels > (uint32_t)MAX_CHANNELS || d->n_rays < 1 || d->n_rays > (uint32_t)MAX_RAYS)
        return false;
    if (!valid_axes(d->f, d->r, d->u)) return false;
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(d->origin[k])) return false;
    for (uint32_t j = 0; j < d->n_channels; ++j) {
        double e = d->elev_rad[j];
        if (!std::isfinite(e) || std::fabs(e) >= M_PI / 2) return false;
        if (j > 0 && !(e > d->elev_rad[j - 1])) return false;
    }
    if (!std::isfinite(d->theta0) || !std::isfinite(d->dtheta) || !(d->dtheta > 0.0)) return false;
    if (d->n_rays * d->dtheta > 2 * M_PI + 1e-9) return false;
    if (std::fabs(d->theta0) > 4 * M_PI) return false;
    if (!(d->d_min >= 0.0) || !(d->d_max >= d->d_min) || !std::isfinite(d->d_min)) return false;
    return true;
}
}  // namespace grca

extern "C" {

const char* grca_status_string(grca_status s) {
    switch (s) {
        case GRCA_OK: return "ok";
        case GRCA_ERR_INVALID_ARG: return "invalid argument";
        case GRCA_ERR_OOM: return "out of memory";
        case GRCA_ERR_CUDA: return "CUDA error";
        case GRCA_ERR_CAPACITY: return "device work queue capacity exceeded";
        case GRCA_ERR_TIMEOUT: return "bounded device wait timed out";
        case GRCA_ERR_NOT_READY: return "not ready (no triangles or sensors)";
        default: return "unknown status";
    }
}

const char* grca_last_cuda_error(grca_ctx* ctx) { return ctx ? ctx->last_err.c_str() : ""; }

grca_status grca_create(grca_ctx** out, int device, const grca_options* opt) {
    if (!out) return GRCA_ERR_INVALID_ARG;
    *out = nullptr;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) return GRCA_ERR_INVALID_ARG;
    grca_ctx* ctx = new (std::nothrow) grca_ctx();
    if (!ctx) return GRCA_ERR_OOM;
    ctx->device = device;
    if (opt) ctx->opt = *opt;
    grca_options& o = ctx->opt;
    if (!o.big_pair_capacity) o.big_pair_capacity = 4u << 20;
    if (!o.chunk_capacity) o.chunk_capacity = 32u << 20;
    if (!o.recheck_capacity) o.recheck_capacity = 8u << 20;
    if (!o.inline_max) o.inline_max = 16;
    if (!o.chunk_rays) o.chunk_rays = 64;
    if (!o.cull_block) o.cull_block = 256;
    if (!o.cull_blocks_per_sm) o.cull_blocks_per_sm = 4;
    if (!o.survivor_capacity) o.survivor_capacity = 256u << 20;
    if (!(o.area_eps > 0.0)) o.area_eps = 1e-6;
    if (o.big_pair_capacity > 0xFFFFFFFFull || o.chunk_capacity > 0xFFFFFFFFull || o.recheck_capacity > 0xFFFFFFFFull ||
        o.survivor_capacity > 0xFFFFFFFFull ||
        o.cull_block % 32 || o.cull_block > 256 || o.cull_block < 32 || o.chunk_rays > 4096) {
        delete ctx;
        return GRCA_ERR_INVALID_ARG;
    }
    ctx->cfg.cull_block = (int)o.cull_block;
    ctx->cfg.cull_blocks_per_sm = (int)o.cull_blocks_per_sm;
    ctx->cfg.inline_max = (int)o.inline_max;
    ctx->cfg.chunk_rays = (int)o.chunk_rays;
    DeviceGuard g(device);
    cudaDeviceProp prop;
    grca_status st = GRCA_OK;
    auto fail = [&](cudaError_t e, const char* w) {
        st = cuda_fail(ctx, e, w);
        return st;
    };
    cudaError_t e;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) fail(e, "cudaGetDeviceProperties");
    if (st == GRCA_OK) ctx->n_sm = prop.multiProcessorCount;
    if (st == GRCA_OK && (e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
        fail(e, "cudaStreamCreate");
    if (st == GRCA_OK && (e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
        fail(e, "cudaStreamCreate");
    if (st == GRCA_OK && (e = cudaEventCreateWithFlags(&ctx->ev_free, cudaEventDisableTiming)) != cudaSuccess)
        fail(e, "cudaEventCreate");
    if (st == GRCA_OK && (e = cudaEventCreateWithFlags(&ctx->ev_copied, cudaEventDisableTiming)) != cudaSuccess)
        fail(e, "cudaEventCreate");
    if (st == GRCA_OK && (e = cudaStreamCreateWithFlags(&ctx->d2h_stream, cudaStreamNonBlocking)) != cudaSuccess)
        fail(e, "cudaStreamCreate");
    if (st == GRCA_OK && (e = cudaEventCreateWithFlags(&ctx->ev_decoded, cudaEventDisableTiming)) != cudaSuccess)
        fail(e, "cudaEventCreate");
    for (int k = 0; k < grca_ctx::OUT_RING && st == GRCA_OK; ++k)
        if ((e = cudaEventCreateWithFlags(&ctx->ev_out[k], cudaEventDisableTiming)) != cudaSuccess)
            fail(e, "cudaEventCreate");
    if (st == GRCA_OK && (e = cudaMalloc(&ctx->d_big, sizeof(BigPair) * o.big_pair_capacity)) != cudaSuccess)
        fail(e, "cudaMalloc(big)");
    if (st == GRCA_OK && (e = cudaMalloc(&ctx->d_setups, sizeof(PairSetup) * o.big_pair_capacity)) != cudaSuccess)
        fail(e, "cudaMalloc(setups)");
    if (st == GRCA_OK && (e = cudaMalloc(&ctx->d_chunks, sizeof(uint4) * o.chunk_capacity)) != cudaSuccess)
        fail(e, "cudaMalloc(chunks)");
    if (st == GRCA_OK && (e = cudaMalloc(&ctx->d_recheck, sizeof(uint4) * o.recheck_capacity)) != cudaSuccess)
        fail(e, "cudaMalloc(recheck)");
    if (st == GRCA_OK && (e = cudaMalloc(&ctx->d_qcount, sizeof(uint32_t) * Q_NUM)) != cudaSuccess)
        fail(e, "cudaMalloc(qcount)");
    if (st == GRCA_OK && (e = cudaMalloc(&ctx->d_counters, sizeof(unsigned long long) * C_NUM)) != cudaSuccess)
        fail(e, "cudaMalloc(counters)");
    if (st == GRCA_OK && (e = cudaMalloc(&ctx->d_error, sizeof(uint32_t))) != cudaSuccess) fail(e, "cudaMalloc(error)");
    if (st == GRCA_OK && (e = cudaMalloc(&ctx->d_sens, sizeof(SensorDev) * MAX_SENSORS)) != cudaSuccess)
        fail(e, "cudaMalloc(sensors)");
    if (st == GRCA_OK && (e = cudaMallocHost(&ctx->h_ring, sizeof(SensorDev) * MAX_SENSORS * RING)) != cudaSuccess)
        fail(e, "cudaMallocHost(ring)");
    for (int k = 0; k < RING; ++k) {
        ctx->ring_used[k] = false;
        if (st == GRCA_OK && (e = cudaEventCreateWithFlags(&ctx->ring_ev[k], cudaEventDisableTiming)) != cudaSuccess)
            fail(e, "cudaEventCreate");
    }
    if (st == GRCA_OK) {
        cudaMemset(ctx->d_qcount, 0, sizeof(uint32_t) * Q_NUM);
        cudaMemset(ctx->d_counters, 0, sizeof(unsigned long long) * C_NUM);
        cudaMemset(ctx->d_error, 0, sizeof(uint32_t));
        cudaDeviceSynchronize();
    }
    if (st != GRCA_OK) {
        grca_destroy(ctx);
        return st;
    }
    *out = ctx;
    return GRCA_OK;
}

void grca_destroy(grca_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    if (ctx->cap_stream) cudaStreamSynchronize(ctx->cap_stream);
    if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
    if (ctx->d2h_stream) cudaStreamSynchronize(ctx->d2h_stream);
    cudaDeviceSynchronize();
    free_graphs(ctx);
    for (SensorHost& sh : ctx->sensors) cudaFree(sh.d_mask);
    cudaFree(ctx->d_tris);
    cudaFree(ctx->d_gb);
    cudaFree(ctx->d_bvh_nodes);
    cudaFree(ctx->d_bvh_prim);
    cudaFree(ctx->d_bvh_tris);
    cudaFree(ctx->d_ch);
    cudaFree(ctx->d_ch64);
    cudaFree(ctx->d_ch_lo);
    cudaFree(ctx->d_az_lo);
    cudaFree(ctx->d_az);
    cudaFree(ctx->d_az64);
    cudaFree(ctx->d_lut);
    cudaFree(ctx->d_keys);
    cudaFree(ctx->d_keys64);
    cudaFree(ctx->d_flag_bits);
    cudaFree(ctx->d_flag_list);
    cudaFree(ctx->d_surv);
    cudaFree(ctx->d_big);
    cudaFree(ctx->d_setups);
    cudaFree(ctx->d_chunks);
    cudaFree(ctx->d_recheck);
    cudaFree(ctx->d_qcount);
    cudaFree(ctx->d_counters);
    cudaFree(ctx->d_error);
    cudaFree(ctx->d_sens);
    cudaFree(ctx->d_out_dist);
    cudaFree(ctx->d_out_tri);
    if (ctx->h_ring) cudaFreeHost(ctx->h_ring);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (int k = 0; k < RING; ++k)
        if (ctx->ring_ev[k]) cudaEventDestroy(ctx->ring_ev[k]);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->ev_free) cudaEventDestroy(ctx->ev_free);
    if (ctx->ev_copied) cudaEventDestroy(ctx->ev_copied);
    if (ctx->d2h_stream) cudaStreamDestroy(ctx->d2h_stream);
    if (ctx->ev_decoded) cudaEventDestroy(ctx->ev_decoded);
    for (cudaEvent_t ev : ctx->ev_out)
        if (ev) cudaEventDestroy(ev);
    delete ctx;
}

grca_status grca_create_sensor(grca_ctx* ctx, const grca_sensor_desc* d, int32_t* out_id) {
    if (!ctx || !out_id || !sensor_desc_valid(d)) return GRCA_ERR_INVALID_ARG;
    SensorHost s;
    s.d = *d;
    s.elev.assign(d->elev_rad, d->elev_rad + d->n_channels);
    s.d.elev_rad = nullptr;
    s.full = std::fabs(d->n_rays * d->dtheta - 2 * M_PI) <= 1e-9;
    ctx->sensors.push_back(std::move(s));
    ctx->tables_dirty = true;
    *out_id = (int32_t)ctx->sensors.size() - 1;
    return GRCA_OK;
}

grca_status grca_set_sensor_pose(grca_ctx* ctx, int32_t id, const double origin[3], const double f[3],
                                 const double r[3], const double u[3]) {
    if (!ctx || !origin || !f || !r || !u || id < 0 || id >= (int32_t)ctx->sensors.size()) return GRCA_ERR_INVALID_ARG;
    if (!valid_axes(f, r, u)) return GRCA_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(origin[k])) return GRCA_ERR_INVALID_ARG;
    grca_sensor_desc& d = ctx->sensors[id].d;
    for (int k = 0; k < 3; ++k) {
        d.origin[k] = origin[k];
        d.f[k] = f[k];
        d.r[k] = r[k];
        d.u[k] = u[k];
    }
    return GRCA_OK;
}

static grca_status copy_in(grca_ctx* ctx, float* dst, const float* src, size_t n_floats, int where,
                           cudaStream_t st) {
    if (n_floats == 0) return GRCA_OK;
    cudaMemcpyKind kind = where == GRCA_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(dst, src, n_floats * sizeof(float), kind, st));
    return GRCA_OK;
}

grca_status grca_upload_triangles(grca_ctx* ctx, const float* xyz, uint32_t n_tris, int where, void* stream) {
    if (!ctx || (!xyz && n_tris) || (where != GRCA_MEM_HOST && where != GRCA_MEM_DEVICE)) return GRCA_ERR_INVALID_ARG;
    if (n_tris > 0x7FFFFFFFu) return GRCA_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (n_tris > ctx->tris_cap) {
        CK(cudaStreamSynchronize(st));
        cudaFree(ctx->d_tris);
        cudaFree(ctx->d_gb);
        ctx->d_tris = nullptr;
        ctx->d_gb = nullptr;
        ctx->tris_cap = 0;
        // + 4 floats of tail padding: the culling pass stages whole float4s
        CK(cudaMalloc(&ctx->d_tris, (9ull * n_tris + 16) * sizeof(float)));
        CK(cudaMemsetAsync(ctx->d_tris, 0, (9ull * n_tris + 16) * sizeof(float), st));
        CK(cudaMalloc(&ctx->d_gb, sizeof(float4) * 2 * ((n_tris + GROUP_TRIS - 1) / GROUP_TRIS + 1)));
        ctx->tris_cap = n_tris;
        free_graphs(ctx);
    }
    ctx->n_tris = n_tris;
    if (ctx->n_static) ctx->bvh_stale = true;  // a new triangle set: rebuild the static hierarchy to use it
    grca_status rs = copy_in(ctx, ctx->d_tris, xyz, 9ull * n_tris, where, st);
    if (rs != GRCA_OK) return rs;
    ctx->gb_lo = 0;
    ctx->gb_hi = n_tris;
    CK(cudaGetLastError());
    return GRCA_OK;
}

grca_status grca_update_vertices(grca_ctx* ctx, const float* xyz, uint32_t first, uint32_t n_tris, int where,
                                 void* stream) {
    if (!ctx || (!xyz && n_tris) || (where != GRCA_MEM_HOST && where != GRCA_MEM_DEVICE)) return GRCA_ERR_INVALID_ARG;
    if ((uint64_t)first + n_tris > ctx->n_tris) return GRCA_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (n_tris && first < ctx->n_static) ctx->bvh_stale = true;  // static triangles moved
    grca_status rs = copy_in(ctx, ctx->d_tris + 9ull * first, xyz, 9ull * n_tris, where, (cudaStream_t)stream);
    if (rs != GRCA_OK) return rs;
    if (n_tris) {
        if (ctx->gb_hi <= ctx->gb_lo) {
            ctx->gb_lo = first;
            ctx->gb_hi = first + n_tris;
        } else {
            ctx->gb_lo = std::min(ctx->gb_lo, first);
            ctx->gb_hi = std::max(ctx->gb_hi, first + n_tris);
        }
    }
    CK(cudaGetLastError());
    return GRCA_OK;
}

grca_status grca_build_static(grca_ctx* ctx, uint32_t n_static, void* stream) {
    if (!ctx || n_static > ctx->n_tris) return GRCA_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(st));
    CK(cudaDeviceSynchronize());  // casts in flight may still read the old hierarchy
    cudaFree(ctx->d_bvh_nodes);
    cudaFree(ctx->d_bvh_prim);
    cudaFree(ctx->d_bvh_tris);
    ctx->d_bvh_nodes = nullptr;
    ctx->d_bvh_prim = nullptr;
    ctx->d_bvh_tris = nullptr;
    ctx->n_static = 0;
    ctx->bvh_stale = false;
    free_graphs(ctx);
    if (n_static == 0) return GRCA_OK;
    std::vector<float> h(9ull * n_static);
    CK(cudaMemcpy(h.data(), ctx->d_tris, sizeof(float) * h.size(), cudaMemcpyDeviceToHost));
    BvhHost bvh;
    if (!build_bvh(h.data(), n_static, bvh)) return GRCA_ERR_CAPACITY;  // tree deeper than the traversal stack
    std::vector<float> leaf(9ull * n_static);
    for (uint32_t k = 0; k < n_static; ++k)
        std::memcpy(&leaf[9ull * k], &h[9ull * bvh.prim[k]], 9 * sizeof(float));
    CK(cudaMalloc(&ctx->d_bvh_nodes, sizeof(BvhNode) * bvh.nodes.size()));
    CK(cudaMalloc(&ctx->d_bvh_prim, sizeof(uint32_t) * n_static));
    CK(cudaMalloc(&ctx->d_bvh_tris, sizeof(float) * leaf.size()));
    CK(cudaMemcpy(ctx->d_bvh_nodes, bvh.nodes.data(), sizeof(BvhNode) * bvh.nodes.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_bvh_prim, bvh.prim.data(), sizeof(uint32_t) * n_static, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_bvh_tris, leaf.data(), sizeof(float) * leaf.size(), cudaMemcpyHostToDevice));
    for (int c = 0; c < 3; ++c) {
        ctx->bvh_lo[c] = bvh.scene_lo[c];
        ctx->bvh_hi[c] = bvh.scene_hi[c];
    }
    ctx->bvh_delta = bvh.delta;
    ctx->n_static = n_static;
    return GRCA_OK;
}

grca_status grca_set_ray_mask(grca_ctx* ctx, int32_t id, const uint32_t* bits, int where, void* stream) {
    if (!ctx || id < 0 || id >= (int32_t)ctx->sensors.size() || (where != GRCA_MEM_HOST && where != GRCA_MEM_DEVICE))
        return GRCA_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    SensorHost& h = ctx->sensors[id];
    cudaStream_t st = (cudaStream_t)stream;
    if (!bits) {
        if (h.d_mask) {
            // casts already queued may still read the mask
            CK(cudaDeviceSynchronize());
            cudaFree(h.d_mask);
            h.d_mask = nullptr;
        }
        return GRCA_OK;
    }
    size_t words = ((size_t)h.d.n_channels * h.d.n_rays + 31) / 32;
    if (!h.d_mask) CK(cudaMalloc(&h.d_mask, sizeof(uint32_t) * words));
    CK(cudaMemcpyAsync(h.d_mask, bits, sizeof(uint32_t) * words,
                       where == GRCA_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (where == GRCA_MEM_HOST) CK(cudaStreamSynchronize(st));
    return GRCA_OK;
}

grca_status grca_set_sensor_azimuths(grca_ctx* ctx, int32_t id, const double* theta) {
    if (!ctx || id < 0 || id >= (int32_t)ctx->sensors.size()) return GRCA_ERR_INVALID_ARG;
    SensorHost& h = ctx->sensors[id];
    if (!theta) {
        if (h.theta.empty()) return GRCA_OK;
        h.theta.clear();
    } else {
        for (uint32_t i = 0; i < h.d.n_rays; ++i) {
            double nominal = h.d.theta0 + (double)i * h.d.dtheta;
            if (!std::isfinite(theta[i]) || !(std::fabs(theta[i] - nominal) < h.d.dtheta)) return GRCA_ERR_INVALID_ARG;
        }
        h.theta.assign(theta, theta + h.d.n_rays);
    }
    ctx->tables_dirty = true;
    return GRCA_OK;
}

grca_status grca_set_range_noise(grca_ctx* ctx, int32_t id, double sigma, uint64_t seed) {
    if (!ctx || id < 0 || id >= (int32_t)ctx->sensors.size() || !std::isfinite(sigma) || !(sigma >= 0.0))
        return GRCA_ERR_INVALID_ARG;
    ctx->sensors[id].range_sigma = sigma;
    ctx->sensors[id].noise_seed = seed;
    return GRCA_OK;
}

grca_status grca_set_debug_dump(grca_ctx* ctx, uint32_t* pairs, uint64_t cap, uint32_t* counter) {
    if (!ctx) return GRCA_ERR_INVALID_ARG;
    if ((pairs == nullptr) != (counter == nullptr) || cap > 0xFFFFFFFFull) return GRCA_ERR_INVALID_ARG;
    ctx->dump = pairs;
    ctx->dump_cap = pairs ? cap : 0;
    ctx->dump_count = counter;
    return GRCA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// cast orchestration
// ---------------------------------------------------------------------------
static grca_status ensure_tables(grca_ctx* ctx, cudaStream_t st) {
    if (!ctx->tables_dirty) return GRCA_OK;
    std::vector<float2> ch;
    std::vector<double2> ch64;
    std::vector<float2> az;
    std::vector<double2> az64;
    std::vector<float2> ch_lo, az_lo;
    std::vector<uint16_t> lut;
    ctx->ch_off.clear();
    ctx->az_off.clear();
    ctx->lut_lo.clear();
    ctx->lut_inv_w.clear();
    for (const SensorHost& s : ctx->sensors) {
        ctx->ch_off.push_back((uint32_t)ch.size());
        std::vector<float> sins;
        for (double e : s.elev) {
            double sn = std::sin(e), cs = std::cos(e);
            ch.push_back(make_float2((float)sn, (float)cs));
            ch64.push_back(make_double2(sn, cs));
            ch_lo.push_back(make_float2((float)(sn - (double)(float)sn), (float)(cs - (double)(float)cs)));
            sins.push_back((float)sn);
        }
        float lo, iw;
        size_t at = lut.size();
        lut.resize(at + LUT_BINS);
        build_channel_lut(sins.data(), (uint32_t)sins.size(), lo, iw, lut.data() + at);
        ctx->lut_lo.push_back(lo);
        ctx->lut_inv_w.push_back(iw);
        ctx->az_off.push_back((uint32_t)az.size());
        for (uint32_t i = 0; i < s.d.n_rays; ++i) {
            double th = s.theta.empty() ? s.d.theta0 + (double)i * s.d.dtheta : s.theta[i];
            double sn = std::sin(th), cs = std::cos(th);
            az.push_back(make_float2((float)sn, (float)cs));
            az64.push_back(make_double2(sn, cs));
            az_lo.push_back(make_float2((float)(sn - (double)(float)sn), (float)(cs - (double)(float)cs)));
        }
    }
    CK(cudaStreamSynchronize(st));
    cudaFree(ctx->d_ch);
    cudaFree(ctx->d_ch64);
    cudaFree(ctx->d_ch_lo);
    cudaFree(ctx->d_az_lo);
    cudaFree(ctx->d_az);
    cudaFree(ctx->d_az64);
    ctx->d_ch = nullptr;
    ctx->d_ch64 = nullptr;
    ctx->d_ch_lo = nullptr;
    ctx->d_az_lo = nullptr;
    ctx->d_az = nullptr;
    ctx->d_az64 = nullptr;
    cudaFree(ctx->d_lut);
    ctx->d_lut = nullptr;
    CK(cudaMalloc(&ctx->d_lut, sizeof(uint16_t) * std::max<size_t>(lut.size(), 1)));
    CK(cudaMemcpy(ctx->d_lut, lut.data(), sizeof(uint16_t) * lut.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_ch, sizeof(float2) * std::max<size_t>(ch.size(), 1)));
    CK(cudaMalloc(&ctx->d_ch64, sizeof(double2) * std::max<size_t>(ch.size(), 1)));
    CK(cudaMalloc(&ctx->d_az, sizeof(float2) * std::max<size_t>(az.size(), 1)));
    CK(cudaMalloc(&ctx->d_az64, sizeof(double2) * std::max<size_t>(az.size(), 1)));
    CK(cudaMemcpy(ctx->d_ch, ch.data(), sizeof(float2) * ch.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_ch64, ch64.data(), sizeof(double2) * ch.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_az, az.data(), sizeof(float2) * az.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_az64, az64.data(), sizeof(double2) * az.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_ch_lo, sizeof(float2) * std::max<size_t>(ch.size(), 1)));
    CK(cudaMalloc(&ctx->d_az_lo, sizeof(float2) * std::max<size_t>(az.size(), 1)));
    CK(cudaMemcpy(ctx->d_ch_lo, ch_lo.data(), sizeof(float2) * ch.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_az_lo, az_lo.data(), sizeof(float2) * az.size(), cudaMemcpyHostToDevice));
    ctx->tables_dirty = false;
    free_graphs(ctx);
    return GRCA_OK;
}

static grca_status ensure_rays(grca_ctx* ctx, size_t n_rays, cudaStream_t st) {
    if (n_rays <= ctx->ray_cap) return GRCA_OK;
    CK(cudaStreamSynchronize(st));
    cudaFree(ctx->d_keys);
    cudaFree(ctx->d_keys64);
    cudaFree(ctx->d_flag_bits);
    cudaFree(ctx->d_flag_list);
    ctx->d_keys = ctx->d_keys64 = nullptr;
    ctx->d_flag_bits = ctx->d_flag_list = nullptr;
    ctx->ray_cap = 0;
    CK(cudaMalloc(&ctx->d_keys, sizeof(unsigned long long) * n_rays));
    CK(cudaMalloc(&ctx->d_keys64, sizeof(unsigned long long) * n_rays));
    CK(cudaMalloc(&ctx->d_flag_bits, sizeof(uint32_t) * ((n_rays + 31) / 32)));
    CK(cudaMalloc(&ctx->d_flag_list, sizeof(uint32_t) * n_rays));
    ctx->ray_cap = n_rays;
    free_graphs(ctx);
    return GRCA_OK;
}

static void fill_sensor(const grca_ctx* ctx, int id, uint32_t ray_off, SensorDev& s) {
    const SensorHost& h = ctx->sensors[id];
    const grca_sensor_desc& d = h.d;
    memset(&s, 0, sizeof(s));
    for (int k = 0; k < 3; ++k) {
        s.o64[k] = d.origin[k];
        s.B64[k] = d.f[k];
        s.B64[3 + k] = d.r[k];
        s.B64[6 + k] = d.u[k];
        float hi = (float)d.origin[k];
        s.o_hi[k] = hi;
        s.o_lo[k] = (float)(d.origin[k] - (double)hi);
    }
    for (int k = 0; k < 9; ++k) {
        s.B[k] = (float)s.B64[k];
        s.B_lo[k] = (float)(s.B64[k] - (double)s.B[k]);
    }
    s.d_min64 = d.d_min;
    s.d_max64 = d.d_max;
    s.theta0 = (float)d.theta0;
    s.dtheta = (float)d.dtheta;
    s.inv_dtheta = (float)(1.0 / d.dtheta);
    s.d_min = (float)d.d_min;
    s.d_max = std::isfinite(d.d_max) ? (float)d.d_max : INFINITY;
    s.period = (float)(2 * M_PI / d.dtheta);
    s.inv_period = 1.0f / (h.full ? (float)d.n_rays : s.period);
    s.n_ch = d.n_channels;
    s.n_rays = d.n_rays;
    s.ch_off = ctx->ch_off[id];
    s.az_off = ctx->az_off[id];
    s.ray_off = ray_off;
    s.full = h.full ? 1u : 0u;
    s.has_range = (d.d_min > 0.0 || std::isfinite(d.d_max)) ? 1u : 0u;
    double det = d.f[0] * (d.r[1] * d.u[2] - d.r[2] * d.u[1]) - d.f[1] * (d.r[0] * d.u[2] - d.r[2] * d.u[0]) +
                 d.f[2] * (d.r[0] * d.u[1] - d.r[1] * d.u[0]);
    s.hand = det < 0.0 ? -1.f : 1.f;
    s.lut_lo = ctx->lut_lo[id];
    s.lut_inv_w = ctx->lut_inv_w[id];
    s.lut_off = (uint32_t)id * LUT_BINS;
    double maxdev = 0.0;
    for (size_t i = 0; i < h.theta.size(); ++i)
        maxdev = std::max(maxdev, std::fabs(h.theta[i] - (d.theta0 + (double)i * d.dtheta)));
    // span widening by the largest perturbation, in ray units, plus rounding slack
    s.az_noise_pad = h.theta.empty() ? 0.f : (float)(maxdev / d.dtheta) + 1e-3f;
    s.mask = h.d_mask;
    s.noise_seed = h.noise_seed;
    s.range_sigma = (float)h.range_sigma;
}

static grca_status prepare_cast(grca_ctx* ctx, const int32_t* ids, uint32_t n, float* out_dist, uint32_t* out_tri,
                                uint32_t flags, cudaStream_t st, CastArgs& a) {
    if (!ids || n < 1 || n > (uint32_t)MAX_SENSORS || !out_dist || !out_tri) return GRCA_ERR_INVALID_ARG;
    if (flags & ~(0xFFu | (uint32_t)GRCA_CAST_NO_OCCLUSION)) return GRCA_ERR_INVALID_ARG;
    if ((flags & GRCA_CAST_DUMP_CANDIDATES) && !ctx->dump) return GRCA_ERR_INVALID_ARG;
    for (uint32_t k = 0; k < n; ++k)
        if (ids[k] < 0 || ids[k] >= (int32_t)ctx->sensors.size()) return GRCA_ERR_INVALID_ARG;
    if (!ctx->d_tris && ctx->n_tris) return GRCA_ERR_NOT_READY;
    grca_status rs = ensure_tables(ctx, st);
    if (rs != GRCA_OK) return rs;
    uint64_t total = 0, total_ch = 0;
    for (uint32_t k = 0; k < n; ++k) {
        const grca_sensor_desc& d = ctx->sensors[ids[k]].d;
        total += (uint64_t)d.n_channels * d.n_rays;
        total_ch += d.n_channels;
    }
    if (total >= 0xFFFFFFFFull || total_ch > 8192) return GRCA_ERR_INVALID_ARG;
    rs = ensure_rays(ctx, total, st);
    if (rs != GRCA_OK) return rs;
    // survivor queue: one slot per (triangle, sensor) pair, capped by the option
    {
        uint64_t need = std::max<uint64_t>((uint64_t)ctx->n_tris * n, 1);
        need = std::min<uint64_t>(need, ctx->opt.survivor_capacity);
        if (need > ctx->surv_cap) {
            CK(cudaStreamSynchronize(st));
            cudaFree(ctx->d_surv);
            ctx->d_surv = nullptr;
            ctx->surv_cap = 0;
            CK(cudaMalloc(&ctx->d_surv, sizeof(unsigned long long) * need));
            ctx->surv_cap = need;
            free_graphs(ctx);
        }
    }
    // stage the descriptors through a pinned ring slot (stream-ordered copy)
    int slot = ctx->ring_pos;
    ctx->ring_pos = (ctx->ring_pos + 1) % RING;
    if (ctx->ring_used[slot]) CK(cudaEventSynchronize(ctx->ring_ev[slot]));
    SensorDev* h = ctx->h_ring + (size_t)slot * MAX_SENSORS;
    uint32_t off = 0, ch_loc = 0;
    for (uint32_t k = 0; k < n; ++k) {
        fill_sensor(ctx, ids[k], off, h[k]);
        h[k].ch_loc = ch_loc;
        off += ctx->sensors[ids[k]].d.n_channels * ctx->sensors[ids[k]].d.n_rays;
        ch_loc += ctx->sensors[ids[k]].d.n_channels;
    }
    uint32_t post = 0;
    for (uint32_t k = 0; k < n; ++k)
        if (h[k].mask || h[k].range_sigma > 0.f) post = 1;
    CK(cudaMemcpyAsync(ctx->d_sens, h, sizeof(SensorDev) * n, cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(ctx->ring_ev[slot], st));
    ctx->ring_used[slot] = true;

    memset(&a, 0, sizeof(a));
    a.tris = ctx->d_tris;
    a.n_tris = ctx->n_tris;
    a.n_sensors = n;
    a.sensors = ctx->d_sens;
    a.ch_sc = ctx->d_ch;
    a.ch_sc64 = ctx->d_ch64;
    a.az_sc = ctx->d_az;
    a.az_sc64 = ctx->d_az64;
    a.ch_lo = ctx->d_ch_lo;
    a.az_lo = ctx->d_az_lo;
    a.lut = ctx->d_lut;
    a.total_ch = (uint32_t)total_ch;
    a.n_rays_total = (uint32_t)total;
    a.keys = ctx->d_keys;
    a.keys64 = ctx->d_keys64;
    a.flag_bits = ctx->d_flag_bits;
    a.flag_list = ctx->d_flag_list;
    a.flag_cap = (uint32_t)ctx->ray_cap;
    a.big_cap = (uint32_t)ctx->opt.big_pair_capacity;
    a.big = ctx->d_big;
    a.setups = ctx->d_setups;
    a.chunks = ctx->d_chunks;
    a.chunk_cap = (uint32_t)ctx->opt.chunk_capacity;
    a.recheck_cap = (uint32_t)ctx->opt.recheck_capacity;
    a.recheck = ctx->d_recheck;
    a.qcount = ctx->d_qcount;
    a.counters = ctx->d_counters;
    a.error = ctx->d_error;
    a.flags = flags;
    a.dump = ctx->dump;
    a.dump_cap = (uint32_t)ctx->dump_cap;
    a.dump_count = ctx->dump_count;
    a.out_dist = out_dist;
    a.out_tri = out_tri;
    a.surv = ctx->d_surv;
    a.surv_cap = (uint32_t)ctx->surv_cap;
    a.area_eps2 = (float)(ctx->opt.area_eps * ctx->opt.area_eps);
    a.post = post;
    // GACP-T_g pays where a range limit empties whole groups; with unlimited
    // range its elevation-only test rarely drops a 32-triangle group and
    // would cost more than it saves, so it runs only when some sensor of the
    // cast has a finite d_max
    bool finite_range = false;
    for (uint32_t k = 0; k < n; ++k) finite_range |= std::isfinite(ctx->sensors[ids[k]].d.d_max);
    a.gbounds = (flags & GRCA_CAST_NO_GROUP_CULL) || !finite_range ? nullptr : ctx->d_gb;
    if (a.gbounds && ctx->gb_hi > ctx->gb_lo && !ctx->defer_bounds) {
        // refresh the boxes of the groups touched since the last refresh (stream-ordered before the cast)
        launch_group_bounds(ctx->d_tris, ctx->n_tris, ctx->gb_lo, ctx->gb_hi - ctx->gb_lo, ctx->d_gb, ctx->n_sm, st);
        CK(cudaGetLastError());
        ctx->pending_launches++;
        ctx->gb_lo = ctx->gb_hi = 0;
    }
    // hybrid: static triangles through the hierarchy when it is current, the
    // mode allows it and every sensor is close enough for its box inflation
    bool hybrid = ctx->d_bvh_nodes && !ctx->bvh_stale && ctx->n_static &&
                  !(flags & (GRCA_CAST_BRUTE | GRCA_CAST_LOSSY_AREA | GRCA_CAST_DUMP_CANDIDATES | GRCA_CAST_NO_STATIC_BVH));
    for (uint32_t k = 0; hybrid && k < n; ++k) {
        const grca_sensor_desc& d = ctx->sensors[ids[k]].d;
        double far2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double e = std::max(std::fabs(ctx->bvh_lo[c] - d.origin[c]), std::fabs(ctx->bvh_hi[c] - d.origin[c]));
            far2 += e * e;
        }
        const double t_far = std::min(std::sqrt(far2), d.d_max);
        if (!(BVH_RAY_ETA * t_far <= ctx->bvh_delta)) hybrid = false;
        // the origin's own coordinates enter the slab rounding as well
        const double omax = std::max(std::fabs(d.origin[0]), std::max(std::fabs(d.origin[1]), std::fabs(d.origin[2])));
        if (!(omax * 0x1p-21 <= 0.5 * ctx->bvh_delta)) hybrid = false;
    }
    if (hybrid) {
        a.tri_first = ctx->n_static;
        a.bvh_nodes = ctx->d_bvh_nodes;
        a.bvh_prim = ctx->d_bvh_prim;
        a.bvh_tris = ctx->d_bvh_tris;
    }
    return GRCA_OK;
}

// launch configurations are tuned per cast shape: sensors, rays, triangles
// through the culls, and the flags that change the work (not GRAPH or DUMP)
static std::tuple<uint32_t, uint32_t, uint32_t, uint32_t> tune_key(const CastArgs& a) {
    return std::make_tuple(a.n_sensors, a.n_rays_total, a.n_tris - a.tri_first,
                           a.flags & (0xE7u | (uint32_t)GRCA_CAST_NO_OCCLUSION));
}

static LaunchCfg cfg_for(grca_ctx* ctx, const CastArgs& a) {
    auto it = ctx->tuned.find(tune_key(a));
    return it == ctx->tuned.end() ? ctx->cfg : it->second;
}

// split_at > 0: launch the key init and the elevation cull of [tri_first,
// split_at) first, wait for `ready` (the copy of the rest), then the rest of
// the frame (graph-replayed when use_graph)
// split_at > 0: part 1 of the frame (key init and the elevation cull of
// triangles below split_at) runs now, then `st` waits for `ready`, then
// `between` (if any) and part 2 are enqueued
static grca_status run_frame(grca_ctx* ctx, CastArgs& a, const LaunchCfg& cfg, cudaStream_t st, bool use_graph,
                             uint32_t split_at = 0, cudaEvent_t ready = nullptr,
                             const std::function<void()>& between = nullptr) {
    a.inline_max = (uint32_t)cfg.inline_max;
    a.chunk_rays = (uint32_t)cfg.chunk_rays;
    uint32_t pending = ctx->pending_launches;
    ctx->pending_launches = 0;
    FrameSplit part2;
    if (split_at) {
        FrameSplit part1;
        part1.part = 1;
        part1.at = split_at;
        KernelMarks mk{profile_mark, ctx};
        pending += (uint32_t)launch_frame(a, cfg, ctx->n_sm, st, ctx->profiling ? &mk : nullptr, part1);
        CK(cudaGetLastError());
        CK(cudaStreamWaitEvent(st, ready, 0));
        if (between) between();
        part2.part = 2;
        part2.at = split_at;
    }
    if (ctx->profiling) {
        KernelMarks mk{profile_mark, ctx};
        ctx->last_launches = pending + (uint32_t)launch_frame(a, cfg, ctx->n_sm, st, &mk, part2);
        CK(cudaGetLastError());
        return GRCA_OK;
    }
    if (!use_graph) {
        ctx->last_launches = pending + (uint32_t)launch_frame(a, cfg, ctx->n_sm, st, nullptr, part2);
        CK(cudaGetLastError());
        return GRCA_OK;
    }
    GraphKey k{a.n_sensors,
               a.n_rays_total,
               a.total_ch,
               a.flags | (a.post ? 0x80000000u : 0u) | (a.gbounds ? 0x40000000u : 0u),
               a.n_tris,
               a.bvh_nodes ? a.tri_first : 0xFFFFFFFFu,
               split_at,
               a.out_dist,
               a.out_tri,
               a.tris,
               a.keys,
               a.dump,
               cfg.cull_block,
               cfg.cull_blocks_per_sm,
               cfg.inline_max,
               cfg.chunk_rays};
    auto it = ctx->graphs.find(k);
    if (it == ctx->graphs.end()) {
        if (ctx->graphs.size() >= 32) free_graphs(ctx);
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        int nl = launch_frame(a, cfg, ctx->n_sm, ctx->cap_stream, nullptr, part2);
        cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
        it = ctx->graphs.emplace(k, std::make_pair(exec, nl)).first;
    }
    ctx->last_launches = pending + (uint32_t)it->second.second;
    CK(cudaGraphLaunch(it->second.first, st));
    return GRCA_OK;
}

extern "C" {

grca_status grca_cast(grca_ctx* ctx, const int32_t* ids, uint32_t n, float* out_dist, uint32_t* out_tri,
                      uint32_t flags, void* stream) {
    if (!ctx) return GRCA_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    CastArgs a;
    grca_status rs = prepare_cast(ctx, ids, n, out_dist, out_tri, flags, st, a);
    if (rs != GRCA_OK) return rs;
    ctx->last_n_rays = a.n_rays_total;
    return run_frame(ctx, a, cfg_for(ctx, a), st, (flags & GRCA_CAST_GRAPH) != 0);
}

grca_status grca_cast_shard(grca_ctx* ctx, const int32_t* ids, uint32_t n, uint32_t tri_base, uint64_t* keys_out,
                            uint32_t flags, void* stream) {
    if (!ctx || !keys_out) return GRCA_ERR_INVALID_ARG;
    if (flags & (GRCA_CAST_GRAPH | GRCA_CAST_BRUTE | GRCA_CAST_DUMP_CANDIDATES | GRCA_CAST_HOST_ASYNC))
        return GRCA_ERR_INVALID_ARG;
    if ((uint64_t)tri_base + ctx->n_tris > 0xFFFFFFFFull) return GRCA_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    CastArgs a;
    // no decode in this stage: the key buffer stands in for the outputs
    grca_status rs = prepare_cast(ctx, ids, n, reinterpret_cast<float*>(keys_out),
                                  reinterpret_cast<uint32_t*>(keys_out), flags, st, a);
    if (rs != GRCA_OK) return rs;
    a.keys_out = reinterpret_cast<unsigned long long*>(keys_out);
    a.tri_base = tri_base;
    const LaunchCfg cfg = cfg_for(ctx, a);
    a.inline_max = (uint32_t)cfg.inline_max;
    a.chunk_rays = (uint32_t)cfg.chunk_rays;
    FrameSplit sp;
    sp.stage = 1;
    ctx->last_n_rays = a.n_rays_total;
    ctx->last_launches = ctx->pending_launches + (uint32_t)launch_frame(a, cfg, ctx->n_sm, st, nullptr, sp);
    ctx->pending_launches = 0;
    CK(cudaGetLastError());
    ctx->shard_args = a;
    ctx->shard_cfg = cfg;
    ctx->shard_ready = true;
    return GRCA_OK;
}

grca_status grca_flag_shard(grca_ctx* ctx, const uint64_t* keys_min, uint8_t* flags_out, void* stream) {
    if (!ctx || !keys_min || !flags_out) return GRCA_ERR_INVALID_ARG;
    if (!ctx->shard_ready) return GRCA_ERR_NOT_READY;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    CastArgs a = ctx->shard_args;
    a.keys_glob = reinterpret_cast<const unsigned long long*>(keys_min);
    a.flags_out = flags_out;
    ctx->shard_args.keys_glob = a.keys_glob;
    FrameSplit sp;
    sp.stage = 2;
    ctx->last_launches = (uint32_t)launch_frame(a, ctx->shard_cfg, ctx->n_sm, st, nullptr, sp);
    CK(cudaGetLastError());
    return GRCA_OK;
}

grca_status grca_resolve_shard(grca_ctx* ctx, const uint8_t* flags_any, uint64_t* keys_out, void* stream) {
    if (!ctx || !flags_any || !keys_out) return GRCA_ERR_INVALID_ARG;
    if (!ctx->shard_ready || !ctx->shard_args.keys_glob) return GRCA_ERR_NOT_READY;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    CastArgs a = ctx->shard_args;
    a.flags_any = flags_any;
    a.keys_out = reinterpret_cast<unsigned long long*>(keys_out);
    FrameSplit sp;
    sp.stage = 3;
    ctx->last_launches = (uint32_t)launch_frame(a, ctx->shard_cfg, ctx->n_sm, st, nullptr, sp);
    CK(cudaGetLastError());
    return GRCA_OK;
}

grca_status grca_decode_keys(grca_ctx* ctx, const uint64_t* keys, float* out_dist, uint32_t* out_tri, void* stream) {
    if (!ctx || !keys || !out_dist || !out_tri) return GRCA_ERR_INVALID_ARG;
    if (!ctx->shard_ready) return GRCA_ERR_NOT_READY;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    CastArgs a = ctx->shard_args;
    a.keys = const_cast<unsigned long long*>(reinterpret_cast<const unsigned long long*>(keys));
    a.out_dist = out_dist;
    a.out_tri = out_tri;
    launch_decode(a, ctx->n_sm, st);
    CK(cudaGetLastError());
    return GRCA_OK;
}

grca_status grca_cast_host(grca_ctx* ctx, const int32_t* ids, uint32_t n, const float* xyz_dyn, uint32_t first_dyn,
                           uint32_t n_dyn, float* out_dist_h, uint32_t* out_tri_h, uint32_t flags, void* stream) {
    if (!ctx || !out_dist_h || !out_tri_h || (!xyz_dyn && n_dyn)) return GRCA_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const bool async_out = flags & GRCA_CAST_HOST_ASYNC;
    flags &= ~(uint32_t)GRCA_CAST_HOST_ASYNC;
    // the copy-out of an earlier asynchronous cast may still read the device
    // result buffers: this frame's decode waits for it (d2h_stream is in order,
    // so the latest copy-out covers the earlier ones)
    auto wait_prev_out = [&]() {
        if (ctx->out_count)
            cudaStreamWaitEvent(st, ctx->ev_out[(ctx->out_head + ctx->out_count - 1) % grca_ctx::OUT_RING], 0);
    };
    // A dynamic tail after a static head: its host-to-device copy runs on the
    // copy stream while the elevation cull works through the static triangles.
    const bool overlap = n_dyn && first_dyn > 0 && (uint64_t)first_dyn + n_dyn == ctx->n_tris &&
                         !(ctx->d_bvh_nodes && !ctx->bvh_stale) && !(flags & GRCA_CAST_BRUTE);
    if (n_dyn && !overlap) {
        grca_status rs = grca_update_vertices(ctx, xyz_dyn, first_dyn, n_dyn, GRCA_MEM_HOST, stream);
        if (rs != GRCA_OK) return rs;
    }
    uint64_t total = 0;
    if (!ids || n < 1 || n > (uint32_t)MAX_SENSORS) return GRCA_ERR_INVALID_ARG;
    for (uint32_t k = 0; k < n; ++k) {
        if (ids[k] < 0 || ids[k] >= (int32_t)ctx->sensors.size()) return GRCA_ERR_INVALID_ARG;
        total += (uint64_t)ctx->sensors[ids[k]].d.n_channels * ctx->sensors[ids[k]].d.n_rays;
    }
    if (total > ctx->out_cap) {
        CK(cudaStreamSynchronize(st));
        CK(cudaStreamSynchronize(ctx->d2h_stream));
        cudaFree(ctx->d_out_dist);
        cudaFree(ctx->d_out_tri);
        ctx->d_out_dist = nullptr;
        ctx->d_out_tri = nullptr;
        ctx->out_cap = 0;
        CK(cudaMalloc(&ctx->d_out_dist, sizeof(float) * total));
        CK(cudaMalloc(&ctx->d_out_tri, sizeof(uint32_t) * total));
        ctx->out_cap = total;
        free_graphs(ctx);
    }
    grca_status rs;
    if (overlap) {
        if (first_dyn < ctx->n_static) ctx->bvh_stale = true;
        // the copy may start once earlier work on `stream` (which may still read
        // the previous frame's vertices) is done
        CK(cudaEventRecord(ctx->ev_free, st));
        CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_free, 0));
        CK(cudaMemcpyAsync(ctx->d_tris + 9ull * first_dyn, xyz_dyn, sizeof(float) * 9ull * n_dyn,
                           cudaMemcpyHostToDevice, ctx->copy_stream));
        CK(cudaEventRecord(ctx->ev_copied, ctx->copy_stream));
        // group boxes of the static head are current unless a stale range
        // from earlier updates reaches below the tail
        const bool head_boxes_current = ctx->gb_hi <= ctx->gb_lo || ctx->gb_lo >= first_dyn;
        if (ctx->gb_hi <= ctx->gb_lo) {
            ctx->gb_lo = first_dyn;
            ctx->gb_hi = first_dyn + n_dyn;
        } else {
            ctx->gb_lo = std::min(ctx->gb_lo, first_dyn);
            ctx->gb_hi = std::max(ctx->gb_hi, first_dyn + n_dyn);
        }
        CastArgs a;
        ctx->defer_bounds = true;
        rs = prepare_cast(ctx, ids, n, ctx->d_out_dist, ctx->d_out_tri, flags, st, a);
        ctx->defer_bounds = false;
        if (rs != GRCA_OK) {
            // the caller may reuse its host buffer once this call returns
            cudaStreamSynchronize(ctx->copy_stream);
            return rs;
        }
        ctx->last_n_rays = a.n_rays_total;
        if (a.gbounds && !a.bvh_nodes && head_boxes_current) {
            // the static head is culled by its (unchanged) group boxes while the
            // tail is copied; the tail's boxes, including a group that straddles
            // the split, are refreshed once the copy is in.  Part 1 reads only
            // static triangles of a straddling group, which its old box bounds.
            const uint32_t lo = ctx->gb_lo, hi = ctx->gb_hi;
            ctx->gb_lo = ctx->gb_hi = 0;
            ctx->pending_launches++;   // the group-bound kernel enqueued between the parts
            rs = run_frame(ctx, a, cfg_for(ctx, a), st, (flags & GRCA_CAST_GRAPH) != 0, first_dyn, ctx->ev_copied,
                           [&]() {
                               wait_prev_out();
                               launch_group_bounds(ctx->d_tris, ctx->n_tris, lo, hi - lo, ctx->d_gb, ctx->n_sm, st);
                           });
        } else if (a.gbounds || a.bvh_nodes) {
            // group boxes (and the hierarchy split) need the new vertices first
            CK(cudaStreamWaitEvent(st, ctx->ev_copied, 0));
            if (a.gbounds && ctx->gb_hi > ctx->gb_lo) {
                launch_group_bounds(ctx->d_tris, ctx->n_tris, ctx->gb_lo, ctx->gb_hi - ctx->gb_lo, ctx->d_gb, ctx->n_sm,
                                    st);
                CK(cudaGetLastError());
                ctx->pending_launches++;
                ctx->gb_lo = ctx->gb_hi = 0;
            }
            wait_prev_out();
            rs = run_frame(ctx, a, cfg_for(ctx, a), st, (flags & GRCA_CAST_GRAPH) != 0);
        } else {
            rs = run_frame(ctx, a, cfg_for(ctx, a), st, (flags & GRCA_CAST_GRAPH) != 0, first_dyn, ctx->ev_copied,
                           wait_prev_out);
        }
    } else {
        wait_prev_out();
        rs = grca_cast(ctx, ids, n, ctx->d_out_dist, ctx->d_out_tri, flags, stream);
    }
    if (rs != GRCA_OK) {
        if (overlap) cudaStreamSynchronize(ctx->copy_stream);   // the host source stays in use until then
        return rs;
    }
    if (async_out) {
        // results go out on d2h_stream while the caller enqueues the next frame;
        // at most OUT_RING casts have copies in flight
        if (ctx->out_count == grca_ctx::OUT_RING) {
            CK(cudaEventSynchronize(ctx->ev_out[ctx->out_head]));
            ctx->out_head = (ctx->out_head + 1) % grca_ctx::OUT_RING;
            ctx->out_count--;
        }
        CK(cudaEventRecord(ctx->ev_decoded, st));
        CK(cudaStreamWaitEvent(ctx->d2h_stream, ctx->ev_decoded, 0));
        CK(cudaMemcpyAsync(out_dist_h, ctx->d_out_dist, sizeof(float) * total, cudaMemcpyDeviceToHost, ctx->d2h_stream));
        CK(cudaMemcpyAsync(out_tri_h, ctx->d_out_tri, sizeof(uint32_t) * total, cudaMemcpyDeviceToHost,
                           ctx->d2h_stream));
        CK(cudaEventRecord(ctx->ev_out[(ctx->out_head + ctx->out_count) % grca_ctx::OUT_RING], ctx->d2h_stream));
        ctx->out_count++;
        return GRCA_OK;
    }
    CK(cudaMemcpyAsync(out_dist_h, ctx->d_out_dist, sizeof(float) * total, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(out_tri_h, ctx->d_out_tri, sizeof(uint32_t) * total, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return GRCA_OK;
}

grca_status grca_host_wait(grca_ctx* ctx, uint32_t max_pending) {
    if (!ctx) return GRCA_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    while (ctx->out_count > max_pending) {
        const cudaError_t e = cudaEventSynchronize(ctx->ev_out[ctx->out_head]);
        ctx->out_head = (ctx->out_head + 1) % grca_ctx::OUT_RING;
        ctx->out_count--;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventSynchronize(copy-out)");
    }
    return GRCA_OK;
}

grca_status grca_get_stats(grca_ctx* ctx, grca_stats* out, void* stream) {
    if (!ctx || !out) return GRCA_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long c[C_NUM];
    uint32_t err = 0;
    CK(cudaMemcpyAsync(c, ctx->d_counters, sizeof(c), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&err, ctx->d_error, sizeof(err), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    memset(out, 0, sizeof(*out));
    out->pairs = c[C_PAIRS];
    out->pairs_live = c[C_PAIRS_LIVE];
    out->survivors = c[C_SURV];
    out->candidates = c[C_CAND];
    out->candidates_inline = c[C_CAND_INLINE];
    out->big_pairs = c[C_BIG];
    out->chunks = c[C_CHUNKS];
    out->tests = c[C_TESTS];
    out->hits = c[C_HITS];
    out->uncertain = c[C_UNCERTAIN];
    out->ties = c[C_TIES];
    out->flagged_rays = c[C_FLAGGED];
    out->recheck_pairs = c[C_RECHECK];
    out->group_culled = c[C_GROUP];
    out->bvh_node_visits = c[C_BVH_VISITS];
    out->bvh_tests = c[C_BVH_TESTS];
    out->n_rays = ctx->last_n_rays;
    out->device_error = err;
    uint64_t* q = &out->queued_edge;
    uint64_t* kp = &out->kept_edge;
    for (int k = 0; k < UC_NUM; ++k) {
        q[k] = c[C_QUEUED0 + k];
        kp[k] = c[C_KEPT0 + k];
    }
    out->t_refined = c[C_REFINED];
    out->pairs_occluded = c[C_OCCLUDED];
    return err ? GRCA_ERR_CAPACITY : GRCA_OK;
}

uint32_t grca_last_launch_count(grca_ctx* ctx) { return ctx ? ctx->last_launches : 0; }

grca_status grca_profile_enable(grca_ctx* ctx, int enable) {
    if (!ctx) return GRCA_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    drain_profile(ctx);
    ctx->profiling = enable != 0;
    for (int k = 0; k < K_NUM; ++k) {
        ctx->total_ms[k] = 0.0;
        ctx->n_launch[k] = 0;
    }
    return GRCA_OK;
}

grca_status grca_profile_read(grca_ctx* ctx, uint32_t max, const char** names, uint64_t* launches, double* total_ms,
                              uint32_t* n_out) {
    if (!ctx || !n_out || (max && (!names || !launches || !total_ms))) return GRCA_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    drain_profile(ctx);
    uint32_t n = std::min<uint32_t>(max, (uint32_t)K_NUM);
    for (uint32_t k = 0; k < n; ++k) {
        names[k] = kKernelNames[k];
        launches[k] = ctx->n_launch[k];
        total_ms[k] = ctx->total_ms[k];
    }
    *n_out = (uint32_t)K_NUM;
    return GRCA_OK;
}

grca_status grca_get_launch_config(grca_ctx* ctx, const int32_t* ids, uint32_t n, uint32_t flags,
                                  int32_t out[4]) {
    if (!ctx || !out) return GRCA_ERR_INVALID_ARG;
    if (!ids || n < 1 || n > (uint32_t)MAX_SENSORS || (flags & ~(0xFFu | (uint32_t)GRCA_CAST_NO_OCCLUSION)))
        return GRCA_ERR_INVALID_ARG;
    uint32_t rays = 0;
    for (uint32_t k = 0; k < n; ++k) {
        if (ids[k] < 0 || ids[k] >= (int32_t)ctx->sensors.size()) return GRCA_ERR_INVALID_ARG;
        rays += ctx->sensors[ids[k]].d.n_channels * ctx->sensors[ids[k]].d.n_rays;
    }
    CastArgs a;
    memset(&a, 0, sizeof(a));
    a.n_sensors = n;
    a.n_rays_total = rays;
    a.n_tris = ctx->n_tris;
    a.flags = flags & ~(uint32_t)(GRCA_CAST_GRAPH | GRCA_CAST_DUMP_CANDIDATES);
    const bool hybrid = ctx->d_bvh_nodes && !ctx->bvh_stale && ctx->n_static &&
                        !(flags & (GRCA_CAST_BRUTE | GRCA_CAST_LOSSY_AREA | GRCA_CAST_DUMP_CANDIDATES | GRCA_CAST_NO_STATIC_BVH));
    a.tri_first = hybrid ? ctx->n_static : 0;
    const LaunchCfg c = cfg_for(ctx, a);
    out[0] = c.inline_max;
    out[1] = c.chunk_rays;
    out[2] = c.cull_block;
    out[3] = c.cull_blocks_per_sm;
    return GRCA_OK;
}

grca_status grca_autotune(grca_ctx* ctx, const int32_t* ids, uint32_t n, float* out_dist, uint32_t* out_tri,
                          uint32_t flags, void* stream, float* out_ms) {
    if (!ctx) return GRCA_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    CastArgs a;
    uint32_t fl = flags & ~(uint32_t)(GRCA_CAST_GRAPH | GRCA_CAST_DUMP_CANDIDATES);
    grca_status rs = prepare_cast(ctx, ids, n, out_dist, out_tri, fl, st, a);
    if (rs != GRCA_OK) return rs;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // one warm-up cast, then the median of 5 timed casts: the minimum of a
    // few casts favoured configurations with one lucky run
    auto time_cfg = [&](const LaunchCfg& c, float& ms) -> grca_status {
        float ts[5];
        for (int rep = 0; rep < 6; ++rep) {
            CastArgs b = a;
            CK(cudaEventRecord(e0, st));
            grca_status r = run_frame(ctx, b, c, st, false);
            if (r != GRCA_OK) return r;
            CK(cudaEventRecord(e1, st));
            CK(cudaEventSynchronize(e1));
            uint32_t err = 0;
            CK(cudaMemcpy(&err, ctx->d_error, sizeof(err), cudaMemcpyDeviceToHost));
            float t;
            CK(cudaEventElapsedTime(&t, e0, e1));
            if (err) t = 1e30f;  // a configuration that overflows a queue is not eligible
            if (rep > 0) ts[rep - 1] = t;
        }
        std::sort(ts, ts + 5);
        ms = ts[2];
        return GRCA_OK;
    };
    LaunchCfg best = cfg_for(ctx, a);
    float best_ms;
    rs = time_cfg(best, best_ms);
    // coordinate descent over the launch parameters
    const int inl[] = {4, 8, 16, 32, 64, 128, 256, 512, 1024};
    const int chk[] = {32, 64, 128, 256};
    const int blk[] = {128, 256};
    const int bps[] = {2, 4, 8, 16, 32};
    for (int pass = 0; pass < 2 && rs == GRCA_OK; ++pass) {
        for (int v : inl) {
            LaunchCfg c = best;
            c.inline_max = v;
            float ms;
            if ((rs = time_cfg(c, ms)) != GRCA_OK) break;
            if (ms < best_ms) best_ms = ms, best = c;
        }
        for (int v : chk) {
            LaunchCfg c = best;
            c.chunk_rays = v;
            float ms;
            if ((rs = time_cfg(c, ms)) != GRCA_OK) break;
            if (ms < best_ms) best_ms = ms, best = c;
        }
        for (int b : blk)
            for (int p : bps) {
                LaunchCfg c = best;
                c.cull_block = b;
                c.cull_blocks_per_sm = p;
                float ms;
                if ((rs = time_cfg(c, ms)) != GRCA_OK) break;
                if (ms < best_ms) best_ms = ms, best = c;
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs != GRCA_OK) return rs;
    ctx->tuned[tune_key(a)] = best;
    if (out_ms) *out_ms = best_ms;
    // leave the outputs holding a valid frame from the chosen configuration
    CastArgs b = a;
    return run_frame(ctx, b, best, st, false);
}

}  // extern "C"
