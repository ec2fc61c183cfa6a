// Internal structures shared by the host runtime (grca_api.cu) and the
// kernels (grca_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "grca.h"

namespace grca {

// host-side argument checks shared by the entry points (grca_api.cu)
bool valid_axes(const double f[3], const double r[3], const double u[3]);
bool sensor_desc_valid(const grca_sensor_desc* d);

// Closest-hit key: (float bits of t) << 32 | triangle id.  For t > 0 the float
// bits order like the floats, so a u64 min is a lexicographic (t, id) min: the
// 64-bit widening of the order-preserving float->u32 map of Sec. A.5.2 (for
// t >= 0 the map is the identity on the bits).  Miss = (+inf, 0xFFFFFFFF).
constexpr unsigned long long KEY_MISS = 0x7F800000FFFFFFFFull;
constexpr uint32_t NO_HIT = 0xFFFFFFFFu;

constexpr int MAX_SENSORS = 64;
constexpr int MAX_CHANNELS = 1024;
constexpr int MAX_RAYS = 32768;

// queue counters (device uint32[8])
// Q_REFINE_N: the re-test queue's length before k_refine, which appends to it
enum { Q_BIG = 0, Q_CHUNK = 1, Q_RECHECK = 2, Q_FLAG = 3, Q_DUMP = 4, Q_SURV = 5, Q_SURV_SPLIT = 6, Q_REFINE_N = 7,
       Q_NUM = 8 };
// statistics counters (device u64[C_NUM])
enum {
    C_PAIRS = 0, C_PAIRS_LIVE, C_CAND, C_CAND_INLINE, C_BIG, C_CHUNKS, C_TESTS, C_HITS,
    C_UNCERTAIN, C_TIES, C_FLAGGED, C_RECHECK, C_SURV, C_GROUP, C_BVH_VISITS, C_BVH_TESTS,
    C_QUEUED0 = 16,   // re-test queue entries per cause (UC_*), C_QUEUED0 + cause
    C_KEPT0 = 21,     // entries per cause kept by the filter (their rays are flagged)
    C_REFINED = 26,   // entries of cause UC_T whose t was re-evaluated in double-float
    C_OCCLUDED = 27,  // live pairs dropped before their setup: every candidate ray already holds a closer hit
    C_NUM = 32
};
// why a (ray, triangle) pair went to the FP64 re-test queue
enum {
    UC_EDGE = 0,    // the ray passes within the FP32 error bound of an edge (|E_k| <= tau_k)
    UC_T = 1,       // inside with margin, but the relative error bound of t exceeds TAU_T
    UC_RANGE = 2,   // t within its error bound of d_min or d_max
    UC_ORIENT = 3,  // |det| within its error bound: facing and orientation unknown
    UC_TIE = 4,     // two certain hits on one ray within the tie band
    UC_NUM = 5
};
// device error bits
enum { ERR_BIG_CAP = 1, ERR_CHUNK_CAP = 2, ERR_RECHECK_CAP = 4, ERR_FLAG_CAP = 8, ERR_DUMP_CAP = 16, ERR_SURV_CAP = 32 };

// One sensor of a cast, as the kernels read it.  FP64 first (alignment).
struct SensorDev {
    double o64[3];
    double B64[9];        // rows f, r, u
    double d_min64, d_max64;
    float o_hi[3], o_lo[3];  // origin = o_hi + o_lo (float pair)
    float B[9];           // rows f, r, u (FP32)
    float B_lo[9];        // B64 - B (FP32): the double-float rotation of the t refinement
    float inv_period;     // 1 / (full ? n_rays : period), correctly rounded
    float theta0, dtheta, inv_dtheta;
    float d_min, d_max;
    float period;         // 2*pi/dtheta, in rays
    uint32_t n_ch, n_rays;
    uint32_t ch_off;      // offset of this sensor's channel table
    uint32_t az_off;      // offset of this sensor's azimuth table
    uint32_t ray_off;     // global ray offset O_n
    uint32_t full;        // 1: the azimuth grid closes the circle (period == n_rays)
    uint32_t has_range;   // 1: d_min > 0 or d_max finite
    uint32_t ch_loc;      // offset of this sensor's channels in the cast-local (shared-memory) table
    float hand;           // det([f; r; u]) = +-1: emitter-frame triple products carry this sign
    float lut_lo;         // channel lookup table: bin b covers sin(elevation) from lut_lo + b / lut_inv_w
    float lut_inv_w;
    uint32_t lut_off;     // offset of this sensor's table in the global lookup-table array
    float az_noise_pad;   // widening of ray spans (ray units) for per-ray azimuth perturbations
    const uint32_t* mask; // on/off bits over the channel x ray grid (nullptr: every ray fires)
    unsigned long long noise_seed;
    float range_sigma;    // post-hoc range noise (0: off)
    uint32_t pad2_;
};

// Channel lookup table: LUT_BINS bins over [sin(elev_0) - 0.01, sin(elev_last) + 0.01];
// bin b stores a channel index no larger than the first channel whose FP32
// sine is >= any value falling in the bin, so a lookup followed by a short
// forward scan gives the exact lower/upper bound in the sorted sine table.
constexpr int LUT_BINS = 512;

inline void build_channel_lut(const float* sins, uint32_t n, float& lo_out, float& inv_w_out, uint16_t* lut) {
    double lo = (double)sins[0] - 0.01, hi = (double)sins[n - 1] + 0.01;
    if (lo < -1.0) lo = -1.0;
    if (hi > 1.0) hi = 1.0;
    double w = (hi - lo) / LUT_BINS;
    lo_out = (float)lo;
    inv_w_out = (float)(1.0 / w);
    uint32_t j = 0;
    for (int b = 0; b < LUT_BINS; ++b) {
        double edge = lo + (b - 0.5) * w;  // half a bin of slack for FP32 rounding of the bin index
        while (j < n && (double)sins[j] < edge) ++j;
        lut[b] = (uint16_t)j;
    }
}

// Per (triangle, sensor) test setup: everything the per-candidate
// ray-triangle test needs (emitter frame), 88 bytes (96 with alignment).
struct __align__(16) PairSetup {
    float m[9];      // folded edge-plane normals: forward hit <=> all d.m_k >= 0
    float tau[3];    // per-edge FP32 error bound of d.m_k
    float n[3];      // emitter-frame normal (v1-v0)x(v2-v0)
    float det;       // (v0-o).n  (world frame); t = det / (d.n)
    float err_det;   // relative FP32 error bound of det
    uint32_t state;  // bit0: |det| within its error bound (facing / orientation uncertain)
    float G[3];      // err(d.n) <= sum_i |d_i| G_i
    float t_lb;      // lower bound of the distance from the origin to any point of the triangle
};

// A (triangle, sensor) pair deferred to the per-channel span pass (32 bytes).
struct __align__(16) BigPair {
    uint32_t tri;
    uint16_t sensor, flags;   // flags bit0: vertical axis pierces (full azimuth)
    uint16_t j_lo, j_hi;      // channel span (inclusive)
    int32_t u_lo;             // first ray of the pair span (unwrapped ray units)
    uint32_t n_r;             // rays in the pair span
    float a0;                 // ray-unit coordinate of vertex 0's azimuth (normalised)
    uint32_t pad_[2];
};

struct Chunk {  // uint4 in memory
    uint32_t bp;      // big pair index
    uint32_t j;       // channel
    uint32_t r0;      // first ray (0..n_rays-1)
    uint32_t count;   // rays (wrapping modulo n_rays)
};

struct CastArgs {
    const float* tris;
    uint32_t n_tris;
    uint32_t n_sensors;
    const SensorDev* sensors;
    const float2* ch_sc;      // (sin, cos) of channel elevations, FP32
    const double2* ch_sc64;
    const float2* az_sc;      // (sin, cos) of ray azimuths, FP32
    const double2* az_sc64;
    const float2* ch_lo;      // FP64 table - FP32 table (low parts): double-float directions
    const float2* az_lo;
    const uint16_t* lut;      // channel lookup tables (LUT_BINS per registered sensor)
    uint32_t total_ch;
    uint32_t n_rays_total;
    unsigned long long* keys;
    unsigned long long* keys64;
    uint32_t* flag_bits;
    uint32_t* flag_list;
    uint32_t flag_cap;
    uint32_t big_cap;
    BigPair* big;
    PairSetup* setups;
    uint4* chunks;
    uint32_t chunk_cap;
    uint32_t recheck_cap;
    uint4* recheck;           // (ray, triangle, bits of a lower bound of t, unused)
    uint32_t* qcount;
    unsigned long long* counters;
    uint32_t* error;
    uint32_t flags;
    uint32_t inline_max;
    uint32_t chunk_rays;
    uint32_t dump_cap;
    uint32_t* dump;           // (ray, tri) pairs
    uint32_t* dump_count;
    float* out_dist;
    uint32_t* out_tri;
    unsigned long long* surv;  // (triangle, sensor, channel span) pairs that pass the elevation cull
    uint32_t surv_cap;
    float area_eps2;           // eps_A^2 of the lossy apparent-area cull (flag bit 5)
    uint32_t post;             // 1: some sensor of the cast has a ray mask or range noise
    const float4* gbounds;     // per 32-triangle group: box lo (xyz, pad), hi (xyz, pad); nullptr: no group cull
    // hybrid static/dynamic pipeline: triangles [0, tri_first) are traced
    // through the static hierarchy, [tri_first, n_tris) go through the culls
    uint32_t tri_first;
    const struct BvhNode* bvh_nodes;  // nullptr: no static hierarchy in this cast
    const uint32_t* bvh_prim;         // leaf order -> triangle id
    const float* bvh_tris;            // vertices in leaf order (9 floats each)
    // survivor pass over part of the queue: 0 all; 1 the survivors queued so
    // far (and record their count); 2 the survivors queued after that
    uint32_t surv_part;
    // elevation pass: the sensors [sens_base, sens_base + sens_count) of this launch
    uint32_t sens_base, sens_count;
    // triangle-sharded casts: this shard's first global triangle id, the
    // per-ray minimum over every shard's FP32 winner (keys_glob), the per-ray
    // flags this shard exports (flags_out) and their maximum over all shards
    // (flags_any), and the output of exported keys
    uint32_t tri_base;
    const unsigned long long* keys_glob;
    uint8_t* flags_out;
    const uint8_t* flags_any;
    unsigned long long* keys_out;
};

struct LaunchCfg {
    int cull_block = 256;
    int cull_blocks_per_sm = 4;
    int inline_max = 16;
    int chunk_rays = 64;
    int test_block = 256;
};

// kernels of one frame, in launch order
enum {
    K_INIT = 0, K_CULL_A, K_CULL_B, K_EXPAND, K_TEST, K_BVH, K_REFINE, K_RECHECK_FILTER, K_RECHECK_RAYS, K_RECHECK_PAIRS,
    K_DECODE,
    K_NUM
};
extern const char* const kKernelNames[K_NUM];

// optional per-kernel hook: called with phase 0 before and phase 1 after each
// kernel launch, on the launching stream (used for CUDA-event timing)
struct KernelMarks {
    void (*fn)(void* user, int kernel, int phase, cudaStream_t st);
    void* user;
};

// launcher (grca_kernels.cu); returns the number of kernels launched
// A frame may be launched in two parts around a wait on the host-to-device
// copy of its dynamic triangles [at, n_tris): part 1 = key init, the
// elevation cull of [tri_first, at) and the survivor pass over its
// survivors; part 2 = the elevation cull of [at, n_tris), the survivor pass
// over the survivors it adds, and everything after.  part 0 = the whole frame.
struct FrameSplit {
    int part = 0;
    uint32_t at = 0;
    // 0: the whole frame; stages of a triangle-sharded cast (triangle ids of
    // exported keys offset by CastArgs::tri_base): 1 the FP32 pass (key init
    // through k_refine) and the keys in keys_out; 2 the filter against
    // keys_glob and the flags in flags_out; 3 the FP64 re-tests of the rays
    // flagged in flags_any and the settled keys in keys_out (no decode)
    int stage = 0;
};
int launch_frame(const CastArgs& a, const LaunchCfg& cfg, int n_sm, cudaStream_t st,
                 const KernelMarks* marks = nullptr, FrameSplit split = FrameSplit());
size_t cull_smem_bytes(const CastArgs& a, const LaunchCfg& cfg);  // fused k_cull
void launch_decode(const CastArgs& a, int n_sm, cudaStream_t st);

// ---------------------------------------------------------------------------
// static hierarchy (hybrid static/dynamic pipeline)
// ---------------------------------------------------------------------------
// A binary node holds both children's boxes (lo xyz, hi xyz) and references:
// >= 0 an inner node, < 0 a leaf of at most BVH_LEAF_MAX triangles in leaf
// order: bit 31 set, first << 3, count - 1 in the low 3 bits.
struct BvhNode {
    float c0lo_x, c0lo_y, c0lo_z, c0hi_x, c0hi_y, c0hi_z;
    float c1lo_x, c1lo_y, c1lo_z, c1hi_x, c1hi_y, c1hi_z;
    int32_t child0, child1, pad0, pad1;
};
static_assert(sizeof(BvhNode) == 64, "one node = four 16-byte loads");
constexpr uint32_t BVH_LEAF_MAX = 8;
constexpr int BVH_STACK = 64;
// Boxes are inflated outward by delta = BVH_ETA * (scene diagonal + 1) +
// 2^-21 * (largest scene coordinate), the last term for the rounding of the
// slab distances.  A
// candidate that the FP32 test can report as a hit or send to the FP64
// re-test lies within ~2e-6 t of the FP32 ray at distance t (table and
// rotation rounding of the direction, the test's error bounds), so the
// traversal is exact for sensors whose farthest scene point is within
// delta / 4e-6 = 1.25 scene diagonals; casts from farther sensors trace the
// static triangles through the culls instead.
constexpr double BVH_ETA = 5e-6;
constexpr double BVH_RAY_ETA = 4e-6;
__host__ __device__ constexpr int32_t bvh_leaf_ref(uint32_t first, uint32_t count) {
    return (int32_t)(0x80000000u | (first << 3) | (count - 1u));
}
struct BvhHost {
    std::vector<BvhNode> nodes;
    std::vector<uint32_t> prim;
    float scene_lo[3] = {0, 0, 0}, scene_hi[3] = {0, 0, 0};
    double delta = 0.0;
    int depth = 0;
};
// host build over n triangles (9 floats each); false if the tree is too deep
bool build_bvh(const float* tris, uint32_t n, BvhHost& out);
void launch_bvh(const CastArgs& a, int n_sm, cudaStream_t st);

// GACP-T_g group bounds: the axis-aligned box of every 32-triangle group that
// overlaps triangles [first, first + n) (lo.xyz, 0 then hi.xyz, 0 per group)
constexpr uint32_t GROUP_TRIS = 32;
void launch_group_bounds(const float* tris, uint32_t n_tris, uint32_t first, uint32_t n, float4* gb, int n_sm,
                         cudaStream_t st);

}  // namespace grca
