// GRCA hot path kernels for sm_103a (GB300).
//
// Per frame (one stream, no host round trip; every kernel reads its work
// count from device memory, so the sequence is capturable as a CUDA graph):
//   k_init     key init (+inf, no id), clear the per-ray flag bits and queue
//              counters (Sec. A.5.1 ray-setup pass).
//   k_cull_a   every (triangle, sensor) pair: group-level cull of 32-triangle
//              tiles (GACP-T_g, Sec. 10.1.1) when a range is set, emitter
//              transform, back-face / range culls (App. A.4.1 Step 1) and the
//              channel span from the exact elevation extent (replaces the
//              binary search of Sec. 3.6); survivors go to a queue, grouped
//              by sensor within each tile.
//   k_cull_b   every survivor, warp-cooperative: azimuth span from the vertex
//              projections (Sec. 3.7), then the pair setup and inline tests of
//              small spans, or an append to the deferred queue (App. A.4.1 Step 4 and A.5.3, BAT
//              list with ballot/popc allocation).
//   k_expand   deferred pairs: per-channel cone/plane crossings give exact
//              per-channel azimuth spans (Sec. 3.5, App. A.4.2 Step 1);
//              rows are cut into fixed-size chunks of a device work queue.
//   k_test     one warp per chunk: watertight FP32 test + closest-hit key.
//   k_bvh      hybrid casts only (Sec. 7): warp-packet traversal of the static
//              hierarchy, committing into the same keys.
//   k_recheck_*  FP64 re-test of every ray the FP32 pass flagged.
//   k_decode   key -> (distance, triangle id) (Sec. A.5.1 output pass), ray
//              masks and range noise (App. A.3, App. A.1).
// k_cull (fused phase A + B) and k_noalloc_prepare serve the allocation-free
// entry point; k_group_bounds runs before a cast that culls by group.
//
// Ray-triangle test.  The paper uses Moller-Trumbore (App. A.4.1 Step 5).
// Here the test is watertight: edge functions E_k = d . (a_k x b_k) of the
// planes through the origin and each edge (a_k, b_k vertices relative to the
// origin, emitter frame).  Each shared edge is evaluated from a canonical
// (lexicographically smaller) base vertex with explicitly rounded arithmetic,
// so two triangles sharing an edge get bitwise-opposite edge functions and no
// ray passes between them.  t = ((v0-o).n) / (d.n).
#include <cooperative_groups.h>
#include <algorithm>
#include <cstddef>
#include <functional>
#include <cmath>
#include <cstring>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "grca_internal.h"

namespace cg = cooperative_groups;

namespace grca {

// ---------------------------------------------------------------------------
// constants of the FP32 pass
// ---------------------------------------------------------------------------
constexpr float U32 = 5.9604645e-08f;   // unit roundoff 2^-24
constexpr float EPS_S = 4e-6f;          // elevation padding (sine space)
constexpr float EPS_T = 4e-6f;          // azimuth padding (radians) + per-vertex term
constexpr float EPS_ROW = 2e-5f;        // per-channel crossing azimuth padding (radians)
constexpr float PADR = 2e-3f;           // ray-unit padding
constexpr float TAU_T = 4e-6f;          // max relative FP32 error of a committed t
constexpr float BETA = 1e-5f;           // tie band (>= 2*TAU_T)

// ---------------------------------------------------------------------------
// explicitly rounded vector helpers: no contraction, bitwise reproducible
// in every kernel that calls them
// ---------------------------------------------------------------------------
struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 vsub(V3 a, V3 b) { return {__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z)}; }
__device__ __forceinline__ float vdot(V3 a, V3 b) {
    return __fmaf_rn(a.x, b.x, __fmaf_rn(a.y, b.y, __fmul_rn(a.z, b.z)));
}
__device__ __forceinline__ V3 vcross(V3 a, V3 b) {
    return {__fsub_rn(__fmul_rn(a.y, b.z), __fmul_rn(a.z, b.y)), __fsub_rn(__fmul_rn(a.z, b.x), __fmul_rn(a.x, b.z)),
            __fsub_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x))};
}
__device__ __forceinline__ V3 vneg(V3 a) { return {-a.x, -a.y, -a.z}; }
__device__ __forceinline__ float vnorm(V3 a) { return sqrtf(vdot(a, a)); }
__device__ __forceinline__ V3 rotB(const float* B, V3 w) {
    return {vdot({B[0], B[1], B[2]}, w), vdot({B[3], B[4], B[5]}, w), vdot({B[6], B[7], B[8]}, w)};
}
__device__ __forceinline__ bool lex_less(V3 a, V3 b) {
    return a.x < b.x || (a.x == b.x && (a.y < b.y || (a.y == b.y && a.z < b.z)));
}
__device__ __forceinline__ float cross2(V3 a, V3 b) { return a.x * b.y - a.y * b.x; }
__device__ __forceinline__ float dot2(V3 a, V3 b) { return a.x * b.x + a.y * b.y; }
// a mod n in [0, n) for n > 0: one period either way without a division
// (the usual case), the division only beyond
__device__ __forceinline__ int imod(int a, int n) {
    int r = a < 0 ? a + n : (a >= n ? a - n : a);
    if ((unsigned)r >= (unsigned)n) {
        r = a % n;
        if (r < 0) r += n;
    }
    return r;
}

// ---------------------------------------------------------------------------
// per-triangle world-frame data (independent of the sensor)
// ---------------------------------------------------------------------------
struct TriW {
    V3 v[3];
    V3 E[3];     // canonical edge vectors V_other - V_base
    int base[3]; // base vertex index of edge k
    float sg[3]; // +1 if the canonical direction follows the winding (k -> k+1)
    V3 n;        // (v1-v0)x(v2-v0)
    V3 N;        // |products| of the cross product terms (error model)
};

__device__ __forceinline__ void tri_world(const float* t9, TriW& T) {
    T.v[0] = {t9[0], t9[1], t9[2]};
    T.v[1] = {t9[3], t9[4], t9[5]};
    T.v[2] = {t9[6], t9[7], t9[8]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int k1 = k == 2 ? 0 : k + 1;
        bool fwd = !lex_less(T.v[k1], T.v[k]);
        T.base[k] = fwd ? k : k1;
        T.sg[k] = fwd ? 1.f : -1.f;
        T.E[k] = fwd ? vsub(T.v[k1], T.v[k]) : vsub(T.v[k], T.v[k1]);
    }
    V3 e1 = vsub(T.v[1], T.v[0]), e2 = vsub(T.v[2], T.v[0]);
    T.n = vcross(e1, e2);
    T.N = {fabsf(e1.y * e2.z) + fabsf(e1.z * e2.y), fabsf(e1.z * e2.x) + fabsf(e1.x * e2.z),
           fabsf(e1.x * e2.y) + fabsf(e1.y * e2.x)};
}

// vertices relative to the origin (world) and in the emitter frame
__device__ __forceinline__ V3 rel_origin(const SensorDev& S, V3 v) {
    return vsub(vsub(v, {S.o_hi[0], S.o_hi[1], S.o_hi[2]}), {S.o_lo[0], S.o_lo[1], S.o_lo[2]});
}

// ---------------------------------------------------------------------------
// test setup of one (triangle, sensor) pair
// ---------------------------------------------------------------------------
// Setup outputs go through a writer: set(k, value) with the field index of
// the setup views below (m 0-8, tau 9-11, n 12-14, det 15, err_det 16,
// state 17, G 18-20, t_lb 21).
struct SetupWriterAoS {
    PairSetup& s;
    __device__ __forceinline__ void set(int k, float v) { reinterpret_cast<float*>(&s)[k] = v; }
};
struct SetupWriterSoA {
    float* base;  // [21][32]
    uint32_t i;
    __device__ __forceinline__ void set(int k, float v) { base[k * 32 + i] = v; }
};

// Hardware approximations in their flush-to-zero forms: the plain forms add
// a rescaling of subnormal inputs and results to every call, which the
// culls pay per pair.  Each call site below stays conservative when a
// subnormal input is taken as zero: rsqrt and rcp then return +inf (a bound
// opens fully), sqrt returns 0 where the bounds' absolute padding covers the
// lost 1e-19, and the operand of rcp_up is clamped into the range where its
// result stays normal, on the side that makes the bound larger.  A NaN input
// stays NaN.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_ftz(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float div_ftz(float a, float b) {
    float r;
    asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
// upper bounds for error-bound arithmetic: hardware approximations (relative
// error <= 2^-22) scaled up by 1 + 2^-18.9; rcp_up of at most 2^126 (so that
// the result stays normal).  sqrt_up keeps the plain form (its flush-to-zero
// form costs k_cull_b a register spill)
__device__ __forceinline__ float sqrt_up(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return __fmul_rn(r, 1.000002f);
}
__device__ __forceinline__ float rcp_up(float x) {
    float r;
    const float xc = x > 8.50705917e37f ? 8.50705917e37f : x;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(xc));
    return __fmul_rn(r, 1.000002f);
}

// Lower bound of the distance from the sensor origin to every point of the
// triangle: each point lies within the longest edge of every vertex, so
// |x - o| >= min_k |p_k| - max_k |p_k1 - p_k|, with p the emitter-frame
// vertices.  Each p_k is within about 7u |p_k| of the exact rotated
// difference (origin split, the FP32 rotation of an orthonormal basis, the
// products), so the edges are within 14u of the farthest vertex's distance;
// the relative padding of 4e-6 covers that, the rounded squares and the
// 2^-22 error of the approximate roots.  Explicitly rounded, so every kernel
// gets the same bits; 0 where the bound is not positive or not finite.
__device__ __forceinline__ float pair_t_lb(const V3 p[3]) {
    const float r2min = fminf(vdot(p[0], p[0]), fminf(vdot(p[1], p[1]), vdot(p[2], p[2])));
    const V3 e0 = vsub(p[1], p[0]), e1 = vsub(p[2], p[1]), e2 = vsub(p[0], p[2]);
    const float ee = fmaxf(vdot(e0, e0), fmaxf(vdot(e1, e1), vdot(e2, e2)));
    const float lb = __fsub_rn(__fmul_rn(sqrt_ftz(r2min), 1.f - 4e-6f), __fmul_rn(sqrt_ftz(ee), 1.f + 4e-6f));
    return lb > 0.f ? lb : 0.f;
}

template <typename WR>
__device__ __forceinline__ void make_setup(const SensorDev& S, const TriW& T, const V3 w[3], const V3 p[3], float det,
                                           float err_det_abs, WR out) {
    out.set(21, pair_t_lb(p));
    bool unc = fabsf(det) <= err_det_abs;
    // forward hit <=> every emitter-frame edge function has the sign of the
    // emitter-frame triple product p0.(p1 x p2) = det(B) * det
    float fold = (det < 0.f ? -1.f : 1.f) * S.hand;
    // every quantity that decides a test outcome is computed with explicitly
    // rounded operations, so that all kernels that set up a pair (culled,
    // deferred and hierarchy paths) get the same bits
    float r2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) r2[k] = vdot(w[k], w[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        V3 e = rotB(S.B, T.E[k]);
        // base vertex by selects (a runtime index would put p[] in local memory)
        const int b = T.base[k];
        const V3 pb = b == 0 ? p[0] : (b == 1 ? p[1] : p[2]);
        const float rb = b == 0 ? r2[0] : (b == 1 ? r2[1] : r2[2]);
        V3 m = vcross(pb, e);
        float f = T.sg[k] * fold;
        if (f < 0.f) m = vneg(m);
        out.set(3 * k + 0, m.x);
        out.set(3 * k + 1, m.y);
        out.set(3 * k + 2, m.z);
        // FP32 error bound of d.m: errors of p_base, e (rotation, origin) and of
        // the cross and dot products, all <= 18 u |p_base| |e| (|m| <= |p_base| |e|)
        const float ee = vdot(T.E[k], T.E[k]);
        out.set(9 + k, __fmaf_rn(18.f * U32, sqrt_up(__fmul_rn(rb, ee)), 1e-30f));
    }
    V3 ne = rotB(S.B, T.n);
    out.set(12, ne.x);
    out.set(13, ne.y);
    out.set(14, ne.z);
    out.set(15, det);
    out.set(16, det != 0.f ? __fmul_rn(err_det_abs, rcp_up(fabsf(det))) : 1.f);
    out.set(17, __uint_as_float(unc ? 1u : 0u));
    const V3 q = {__fmul_rn(3.f, __fadd_rn(fabsf(T.n.x), T.N.x)), __fmul_rn(3.f, __fadd_rn(fabsf(T.n.y), T.N.y)),
                  __fmul_rn(3.f, __fadd_rn(fabsf(T.n.z), T.N.z))};
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const V3 br = {fabsf(S.B[3 * r]), fabsf(S.B[3 * r + 1]), fabsf(S.B[3 * r + 2])};
        const float ner = r == 0 ? ne.x : (r == 1 ? ne.y : ne.z);
        out.set(18 + r, __fmul_rn(U32, __fmaf_rn(6.f, fabsf(ner), vdot(br, q))));
    }
}

// FP32 error bound of det = w0.n used by the back-face cull (n = (v1-v0)x(v2-v0),
// N the sums of |products| of its cross-product terms)
__device__ __forceinline__ float backface_err(const V3& w0, const V3& n, const V3& N) {
    const V3 aw = {fabsf(w0.x), fabsf(w0.y), fabsf(w0.z)};
    const V3 c = {__fmaf_rn(3.f, N.x, __fmul_rn(4.f, fabsf(n.x))), __fmaf_rn(3.f, N.y, __fmul_rn(4.f, fabsf(n.y))),
                  __fmaf_rn(3.f, N.z, __fmul_rn(4.f, fabsf(n.z)))};
    return __fmul_rn(U32, vdot(aw, c));
}

__device__ __forceinline__ float det_error(const V3& w0, const TriW& T) {
    return __fadd_rn(backface_err(w0, T.n, T.N), 1e-35f);
}

// ---------------------------------------------------------------------------
// per-candidate test
// ---------------------------------------------------------------------------
// T_UNCERTAIN + cause: the FP32 result needs the FP64 re-test (recheck mode
// only); the cause (UC_*) goes with the queued entry for the statistics
enum { T_MISS = 0, T_HIT = 1, T_UNCERTAIN = 2 };
__device__ __forceinline__ bool is_uncertain(int res) { return res >= T_UNCERTAIN; }

__device__ __forceinline__ V3 ray_dir(float2 ch, float2 az) {
    // Eq. ray_dir in the emitter frame: (cos th cos ph, sin th cos ph, sin ph); (x=sin, y=cos)
    return {__fmul_rn(az.y, ch.y), __fmul_rn(az.x, ch.y), ch.x};
}

// FP32 test.  Plain mode: inclusive edge test, T_HIT or T_MISS.  Recheck mode
// additionally returns T_UNCERTAIN when the FP32 decision or t is not
// guaranteed; *t_err receives the relative error bound of t.
// A pair setup is read through a view: the PairSetup struct itself, or one
// lane's column of a field-major shared-memory copy (conflict-free).
// Field index: m 0-8, tau 9-11, n 12-14, det 15, err_det 16, state 17, G 18-20,
// distance lower bound 21.
constexpr int SETUP_FIELDS = 22;
static_assert(offsetof(PairSetup, tau) == 9 * 4 && offsetof(PairSetup, n) == 12 * 4 && offsetof(PairSetup, det) == 15 * 4 &&
                  offsetof(PairSetup, err_det) == 16 * 4 && offsetof(PairSetup, state) == 17 * 4 &&
                  offsetof(PairSetup, G) == 18 * 4 && offsetof(PairSetup, t_lb) == 21 * 4,
              "setup field indices");
struct SetupAoS {
    const PairSetup& s;
    __device__ __forceinline__ float f(int k) const { return reinterpret_cast<const float*>(&s)[k]; }
};
struct SetupSoA {
    const float* base;  // [SETUP_FIELDS][32]
    uint32_t i;
    __device__ __forceinline__ float f(int k) const { return base[k * 32 + i]; }
};

struct SetupReg {
    float f_[SETUP_FIELDS];
    __device__ __forceinline__ float f(int k) const { return f_[k]; }
};
struct SetupWriterReg {
    SetupReg& r;
    __device__ __forceinline__ void set(int k, float v) { r.f_[k] = v; }
};

template <bool RECHECK, typename SV>
__device__ __forceinline__ int test_fp32(const SV& st, const SensorDev& S, V3 d, float& t, float& t_err) {
    V3 m0 = {st.f(0), st.f(1), st.f(2)}, m1 = {st.f(3), st.f(4), st.f(5)}, m2 = {st.f(6), st.f(7), st.f(8)};
    float E0 = vdot(d, m0), E1 = vdot(d, m1), E2 = vdot(d, m2);
    float dn = vdot(d, {st.f(12), st.f(13), st.f(14)});
    // t = det / dn through one correctly rounded reciprocal (also used by the
    // error bound); t then carries <= 1 ulp more error than a division
    const float rdn = __frcp_rn(dn);
    t = __fmul_rn(st.f(15), rdn);
    t_err = 0.f;
    if (!RECHECK) {
        if (E0 < 0.f || E1 < 0.f || E2 < 0.f) return T_MISS;
        if (!(t > 0.f) || !(t <= S.d_max) || t < S.d_min) return T_MISS;
        return T_HIT;
    }
    const float tau0 = st.f(9), tau1 = st.f(10), tau2 = st.f(11);
    bool unc_pair = __float_as_uint(st.f(17)) & 1u;
    if (E0 < -tau0 || E1 < -tau1 || E2 < -tau2) {
        if (!unc_pair) return T_MISS;
        // orientation unknown: the other orientation may still hold
        if (E0 <= tau0 && E1 <= tau1 && E2 <= tau2) {
            t_err = 1.f;
            return T_UNCERTAIN + UC_ORIENT;
        }
        return T_MISS;
    }
    bool inside = E0 > tau0 && E1 > tau1 && E2 > tau2;
    t_err = __fadd_rn(__fmaf_rn(vdot({fabsf(d.x), fabsf(d.y), fabsf(d.z)}, {st.f(18), st.f(19), st.f(20)}), fabsf(rdn),
                                st.f(16)),
                      2.4e-7f);
    // cause of an uncertain result, first that applies: orientation, edge, range, t
    const int unc_base = T_UNCERTAIN + (unc_pair ? UC_ORIENT : (!inside ? UC_EDGE : UC_T));
    if (!(t > 0.f) || !(t_err < 0.25f)) {
        t_err = 1.f;
        return (inside && !unc_pair && !(t > 0.f)) ? T_MISS : unc_base;
    }
    if (S.has_range) {
        const float lo = __fmul_rn(t, __fsub_rn(1.f, t_err)), hi = __fmul_rn(t, __fadd_rn(1.f, t_err));
        if (hi < S.d_min || lo > S.d_max) return T_MISS;
        if (lo < S.d_min || hi > S.d_max) return (inside && !unc_pair) ? T_UNCERTAIN + UC_RANGE : unc_base;
    }
    if (!inside || unc_pair || t_err > TAU_T) return unc_base;
    return T_HIT;
}

// ---------------------------------------------------------------------------
// closest-hit commit, flags and the re-test queue
// ---------------------------------------------------------------------------
__device__ __forceinline__ void flag_ray(const CastArgs& a, uint32_t g) {
    uint32_t bit = 1u << (g & 31u);
    uint32_t old = atomicOr(&a.flag_bits[g >> 5], bit);
    if (!(old & bit)) {
        uint32_t idx = atomicAdd(&a.qcount[Q_FLAG], 1u);
        if (idx < a.flag_cap)
            a.flag_list[idx] = g;
        else
            atomicOr(a.error, (uint32_t)ERR_FLAG_CAP);
    }
}

// queue (ray, triangle, lower bound of t) for the FP64 re-test; the filter
// pass keeps it only if it can still beat or tie the ray's final FP32 winner
__device__ __forceinline__ void push_recheck(const CastArgs& a, uint32_t g, uint32_t tri, float t_lo, uint32_t cause) {
    uint32_t idx = atomicAdd(&a.qcount[Q_RECHECK], 1u);
    if (idx < a.recheck_cap)
        a.recheck[idx] = make_uint4(g, tri, __float_as_uint(t_lo), cause);
    else
        atomicOr(a.error, (uint32_t)ERR_RECHECK_CAP);
}

// An uncertain FP32 result goes to the re-test queue with a lower bound of
// its distance: t (1 - t_err) where that error bound is usable, raised to the
// pair's distance lower bound t_lb (0 where none is known).  It is not queued
// when that bound lies beyond the tie band of the ray's current best hit: the
// filter would drop it against the final winner, which is no farther.
// Returns 1 if queued.
__device__ __forceinline__ uint32_t queue_uncertain(const CastArgs& a, uint32_t g, uint32_t tri, int res, float t,
                                                    float t_err, float t_lb, float tcur) {
    const bool t_ok = t_err < 0.25f && t > 0.f;
    const float t_lo = t_ok ? fmaxf(__fmul_rn(t, __fsub_rn(1.f, t_err)), t_lb) : t_lb;
    if (t_lo > __fmul_rn(tcur, 1.f + BETA)) return 0u;
    push_recheck(a, g, tri, t_lo, (uint32_t)(res - T_UNCERTAIN));
    return 1u;
}

__device__ __noinline__ void dump_candidate(const CastArgs& a, uint32_t g, uint32_t tri) {
    uint32_t idx = atomicAdd(a.dump_count, 1u);
    if (idx < a.dump_cap) {
        a.dump[2 * idx] = g;
        a.dump[2 * idx + 1] = tri;
    } else {
        atomicOr(a.error, (uint32_t)ERR_DUMP_CAP);
    }
}

// ---------------------------------------------------------------------------
// double-float arithmetic: a value h + l held in two FP32, explicitly rounded
// (Knuth's two-sum, the FMA two-product and their usual combinations).
// Error bounds below use u = 2^-24 and normalised inputs (|l| <= u |h|).
// ---------------------------------------------------------------------------
struct DF {
    float h, l;
};
__device__ __forceinline__ DF two_sum(float a, float b) {  // exact: h + l = a + b
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF two_prod(float a, float b) {  // exact: h + l = a * b
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_norm(float h, float e) {
    const float s = __fadd_rn(h, e);
    return {s, __fsub_rn(e, __fsub_rn(s, h))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {  // |error| <= 8 u^2 (|x| + |y|)
    const DF s = two_sum(x.h, y.h);
    return df_norm(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ DF df_sub(DF x, DF y) { return df_add(x, DF{-y.h, -y.l}); }
__device__ __forceinline__ DF df_mul(DF x, DF y) {  // |error| <= 8 u^2 |x| |y|
    const DF p = two_prod(x.h, y.h);
    return df_norm(p.h, __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, p.l)));
}

// Re-evaluation of t for a candidate whose FP32 test is certain about the hit
// (inside every edge with margin, facing known) but whose FP32 distance has
// an error bound above TAU_T: grazing incidence, where d.n cancels.  t =
// ((v0 - o).n) / (D.n) in the world frame, in double-float from the FP32
// vertices (differences exact), the origin o_hi + o_lo, the direction D =
// B^T d from the FP64 tables as high + low parts and B as B + B_lo.  Bounds
// from the operation bounds above: |err(n_c)| <= 16 u^2 N_c (N_c the sum of
// the two products' magnitudes), |err(w0_c)| <= 10 u^2 (|w0_c| + |o_c|),
// |err(det)| <= 34 u^2 M_det, |err(D_c)| <= 64 u^2, |err(D.n)| <= 88 u^2 M_dn,
// M_det = sum_c |w0_c| (|n_c| + N_c) + |o_c| |n_c|, M_dn = sum_c |n_c| + N_c;
// the relative bound of t adds both relative terms (taken 1.5 times) and the
// final rounding to FP32.  Returns T_HIT (t, t_err refined), T_MISS, or
// T_UNCERTAIN + cause (t, t_err unchanged unless the cause is the range).
struct Refined {
    int res;
    float t, e;
};
__device__ __noinline__ Refined refine_t(const CastArgs& a, const SensorDev& S, uint32_t j, uint32_t i, uint32_t tri) {
    const float* t9 = a.tris + 9ull * tri;
    const float v0x = __ldg(t9 + 0), v0y = __ldg(t9 + 1), v0z = __ldg(t9 + 2);
    const DF e1x = two_sum(__ldg(t9 + 3), -v0x), e1y = two_sum(__ldg(t9 + 4), -v0y), e1z = two_sum(__ldg(t9 + 5), -v0z);
    const DF e2x = two_sum(__ldg(t9 + 6), -v0x), e2y = two_sum(__ldg(t9 + 7), -v0y), e2z = two_sum(__ldg(t9 + 8), -v0z);
    const DF nx = df_sub(df_mul(e1y, e2z), df_mul(e1z, e2y));
    const DF ny = df_sub(df_mul(e1z, e2x), df_mul(e1x, e2z));
    const DF nz = df_sub(df_mul(e1x, e2y), df_mul(e1y, e2x));
    const float Nx = fabsf(e1y.h * e2z.h) + fabsf(e1z.h * e2y.h), Ny = fabsf(e1z.h * e2x.h) + fabsf(e1x.h * e2z.h),
                Nz = fabsf(e1x.h * e2y.h) + fabsf(e1y.h * e2x.h);
    const DF wx = df_add(two_sum(v0x, -S.o_hi[0]), DF{-S.o_lo[0], 0.f});
    const DF wy = df_add(two_sum(v0y, -S.o_hi[1]), DF{-S.o_lo[1], 0.f});
    const DF wz = df_add(two_sum(v0z, -S.o_hi[2]), DF{-S.o_lo[2], 0.f});
    const DF det = df_add(df_add(df_mul(wx, nx), df_mul(wy, ny)), df_mul(wz, nz));
    // emitter-frame direction (cos th cos ph, sin th cos ph, sin ph), then D = B^T d
    const float2 ch = __ldg(&a.ch_sc[S.ch_off + j]), chl = __ldg(&a.ch_lo[S.ch_off + j]);
    const float2 az = __ldg(&a.az_sc[S.az_off + i]), azl = __ldg(&a.az_lo[S.az_off + i]);
    const DF cph = {ch.y, chl.y};
    const DF d0 = df_mul(DF{az.y, azl.y}, cph), d1 = df_mul(DF{az.x, azl.x}, cph), d2 = {ch.x, chl.x};
    DF D[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        D[c] = df_add(df_add(df_mul(d0, DF{S.B[c], S.B_lo[c]}), df_mul(d1, DF{S.B[3 + c], S.B_lo[3 + c]})),
                      df_mul(d2, DF{S.B[6 + c], S.B_lo[6 + c]}));
    const DF dn = df_add(df_add(df_mul(D[0], nx), df_mul(D[1], ny)), df_mul(D[2], nz));
    const float m_det = fabsf(wx.h) * (fabsf(nx.h) + Nx) + fabsf(wy.h) * (fabsf(ny.h) + Ny) +
                        fabsf(wz.h) * (fabsf(nz.h) + Nz) +
                        (fabsf(S.o_hi[0]) * fabsf(nx.h) + fabsf(S.o_hi[1]) * fabsf(ny.h) + fabsf(S.o_hi[2]) * fabsf(nz.h));
    const float m_dn = fabsf(nx.h) + Nx + fabsf(ny.h) + Ny + fabsf(nz.h) + Nz;
    constexpr float U2 = U32 * U32;
    const float e = 1.02f * (51.f * U2 * m_det / fabsf(det.h) + 132.f * U2 * m_dn / fabsf(dn.h)) + 3.1e-8f;
    Refined r{T_UNCERTAIN + UC_T, 0.f, 0.f};
    if (!(e <= TAU_T)) return r;  // also NaN / zero det or dn
    // t = det / dn: correctly rounded quotient of the high parts, one
    // correction from the exact remainder
    const float q = __fdiv_rn(det.h, dn.h);
    const float rem = __fadd_rn(__fmaf_rn(-q, dn.h, det.h), __fmaf_rn(-q, dn.l, det.l));
    const float t = __fadd_rn(q, __fdiv_rn(rem, dn.h));
    if (!(t > 0.f)) {
        r.res = T_MISS;
        return r;
    }
    r.t = t;
    r.e = e;
    r.res = T_HIT;
    if (S.has_range) {
        const float lo = __fmul_rn(t, __fsub_rn(1.f, e)), hi = __fmul_rn(t, __fadd_rn(1.f, e));
        if (hi < S.d_min || lo > S.d_max) r.res = T_MISS;
        else if (lo < S.d_min || hi > S.d_max) r.res = T_UNCERTAIN + UC_RANGE;
    }
    return r;
}

// Closest-hit commit.  Certain FP32 hits go into the u64 key with
// atomicMin (after a plain L2 load that skips hits that cannot win); in the
// recheck mode two certain hits on one ray within the tie band queue both
// triangles, and uncertain tests queue theirs, for the FP64 re-test.
// Returns 1 if a hit was committed (for the statistics).
template <bool RECHECK>
__device__ __forceinline__ int commit_pre(const CastArgs& a, uint32_t g, uint32_t tri, int res, float t, float t_err,
                                          float t_lb, unsigned long long cur, uint32_t& n_unc, uint32_t& n_ties) {
    if (res == T_MISS) return 0;
    unsigned long long* kp = &a.keys[g];
    float tcur = __uint_as_float((uint32_t)(cur >> 32));
    if (is_uncertain(res)) {
        // a re-test can only change the result if it may beat the current best
        n_unc += queue_uncertain(a, g, tri, res, t, t_err, t_lb, tcur);
        return 0;
    }
    unsigned long long key = ((unsigned long long)__float_as_uint(t) << 32) | tri;
    if (!RECHECK) {
        if (key < cur) atomicMin(kp, key);
        return 1;
    }
    if (t > __fmul_rn(tcur, 1.f + BETA)) return 1;
    unsigned long long old = atomicMin(kp, key);
    uint32_t oid = (uint32_t)old;
    if (oid != NO_HIT && oid != tri) {
        float told = __uint_as_float((uint32_t)(old >> 32));
        if (fabsf(__fsub_rn(t, told)) <= __fmul_rn(BETA, fmaxf(t, told))) {
            push_recheck(a, g, tri, __fmul_rn(t, 1.f - TAU_T), UC_TIE);
            push_recheck(a, g, oid, __fmul_rn(told, 1.f - TAU_T), UC_TIE);
            n_ties++;
        }
    }
    return 1;
}

template <bool RECHECK>
__device__ __forceinline__ int commit(const CastArgs& a, uint32_t g, uint32_t tri, int res, float t, float t_err,
                                      float t_lb, uint32_t& n_unc, uint32_t& n_ties) {
    if (res == T_MISS) return 0;
    return commit_pre<RECHECK>(a, g, tri, res, t, t_err, t_lb, __ldcg(&a.keys[g]), n_unc, n_ties);
}

// ---------------------------------------------------------------------------
// spans
// ---------------------------------------------------------------------------
struct Span {
    int j_lo, j_hi;
    int u_lo, n_r;  // ray span: unwrapped first ray and count
    float a0;       // ray-unit coordinate of vertex 0's azimuth (normalised)
    bool pierced;
};

// elevation extremum inside edge a->b (see Sec. 3.5.2 for the cone/edge
// quadratic; here: the extreme elevation of the great-circle arc of the edge)
__device__ __forceinline__ void edge_elev_extremum(V3 a, V3 b, float& smin, float& smax) {
    V3 e = {b.x - a.x, b.y - a.y, b.z - a.z};
    float ae = a.x * e.x + a.y * e.y + a.z * e.z;
    float aa = a.x * a.x + a.y * a.y + a.z * a.z;
    float ee = e.x * e.x + e.y * e.y + e.z * e.z;
    float num = a.z * ae - e.z * aa;
    float den = e.z * ae - a.z * ee;
    if (den < 0.f) {
        num = -num;
        den = -den;
    }
    // lambda* = num/den must lie in (-1e-3, 1.001) (padded edge interior)
    if (!(den > 0.f) || !(num > -1e-3f * den) || !(num < 1.001f * den)) return;
    V3 m = {a.y * e.z - a.z * e.y, a.z * e.x - a.x * e.z, a.x * e.y - a.y * e.x};
    float mh = m.x * m.x + m.y * m.y;
    float mm = mh + m.z * m.z;
    if (!(mm > 1e-12f * aa * ee)) return;  // edge collinear with the origin: vertices bound it
    float v = sqrtf(mh * __frcp_rn(mm));
    float lam = fminf(fmaxf(num / den, 0.f), 1.f);
    float qz = a.z + lam * e.z;
    float tol = 1e-4f * sqrtf(aa + ee);
    if (qz >= -tol) smax = fmaxf(smax, v);
    if (qz <= tol) smin = fminf(smin, -v);
}

__device__ __forceinline__ int lower_bound_sin(const float2* ch, int n, float x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (ch[mid].x < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int upper_bound_sin(const float2* ch, int n, float x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (ch[mid].x <= x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// ray-unit coordinate of an absolute azimuth, normalised into one period
__device__ __forceinline__ float ray_units(const SensorDev& S, float theta) {
    float x = (theta - S.theta0) * S.inv_dtheta;
    // normalise into one period [g0, g0 + P); P = n_rays for full circles
    float P = S.full ? (float)S.n_rays : S.period;
    float g0 = S.full ? 0.f : -0.5f * (S.period - (float)S.n_rays);
    x -= P * floorf((x - g0) * S.inv_period);
    return x;
}

// integer rays in [A, B] (ray units, around the normalised a0); wrap for
// full circles, clip to the field of view otherwise
__device__ __forceinline__ bool ray_interval(const SensorDev& S, float A, float B, int& u_lo, int& n_r) {
    int n = (int)S.n_rays;
    if (S.full) {
        int ia = (int)ceilf(A), ib = (int)floorf(B);
        if (ib < ia) return false;
        int cnt = ib - ia + 1;
        if (cnt >= n) {
            u_lo = 0;
            n_r = n;
        } else {
            u_lo = ia;
            n_r = cnt;
        }
        return true;
    }
    int lo = n, hi = -1;
    float P = S.period;
#pragma unroll
    for (int s = -1; s <= 1; ++s) {
        int ia = (int)ceilf(A + s * P), ib = (int)floorf(B + s * P);
        ia = max(ia, 0);
        ib = min(ib, n - 1);
        if (ia <= ib) {
            lo = min(lo, ia);
            hi = max(hi, ib);
        }
    }
    if (hi < lo) return false;
    u_lo = lo;
    n_r = hi - lo + 1;
    return true;
}

// azimuth padding of a direction: FP32 errors of p scale with |p|, so the
// azimuth error scales with |p| / |p_h| = 1 / sqrt(1 - sin^2(elevation))
__device__ __forceinline__ float az_pad_s(float s) {
    float c2 = 1.f - s * s;
    return c2 > 1e-12f ? 16.f * U32 * rsqrtf(c2) : 10.f;
}
__device__ __forceinline__ float az_pad(V3 p) {
    float h2 = p.x * p.x + p.y * p.y;
    float r2 = h2 + p.z * p.z;
    return h2 > 1e-12f * r2 ? 16.f * U32 * sqrtf(r2 / h2) : 10.f;
}

__device__ __forceinline__ float fast_atan2(float y, float x);

// angle from a to b in the xy plane, in (-pi, pi]; small angles by the
// series atan(x) = x - x^3/3 + x^5/5 (error < x^7/7 < 2e-12 for |x| < 0.02),
// larger ones by fast_atan2 (error < FAST_ATAN_PAD)
__device__ __forceinline__ float rel_angle(V3 a, V3 b) {
    float cr = cross2(a, b), dt = dot2(a, b);
    if (dt >= 1.17549435e-38f && fabsf(cr) < 0.02f * dt) {
        // |x| < 0.02; the fast division's 2-ulp error adds < 1e-8 rad
        float x = div_ftz(cr, dt), x2 = x * x;
        return x * (1.f - x2 * (0.33333334f - 0.2f * x2));
    }
    return fast_atan2(cr, dt);  // callers pad by FAST_ATAN_PAD per call
}

// Does the vertical axis through the origin meet the triangle?  Point in the
// xy-projection, closed, with a margin of 1e-5 |p| plus the FP32 error of the
// 2-D edge functions.  The bounding-box test keeps triangles whose projection
// degenerates to a segment (vertical faces seen edge-on) from passing on the
// edge functions alone.
__device__ __forceinline__ bool axis_pierces(const V3 p[3]) {
    float q0 = p[0].x * p[0].x + p[0].y * p[0].y, q1 = p[1].x * p[1].x + p[1].y * p[1].y,
          q2 = p[2].x * p[2].x + p[2].y * p[2].y;
    float dm = 1e-5f * sqrtf(fmaxf(q0, fmaxf(q1, q2)));
    float mnx = fminf(p[0].x, fminf(p[1].x, p[2].x)), mxx = fmaxf(p[0].x, fmaxf(p[1].x, p[2].x));
    float mny = fminf(p[0].y, fminf(p[1].y, p[2].y)), mxy = fmaxf(p[0].y, fmaxf(p[1].y, p[2].y));
    if (mnx > dm || mxx < -dm || mny > dm || mxy < -dm) return false;
    float c0 = cross2(p[0], p[1]), c1 = cross2(p[1], p[2]), c2 = cross2(p[2], p[0]);
    float t0 = dm * (fabsf(p[1].x - p[0].x) + fabsf(p[1].y - p[0].y)) + 16.f * U32 * (q0 + q1);
    float t1 = dm * (fabsf(p[2].x - p[1].x) + fabsf(p[2].y - p[1].y)) + 16.f * U32 * (q1 + q2);
    float t2 = dm * (fabsf(p[0].x - p[2].x) + fabsf(p[0].y - p[2].y)) + 16.f * U32 * (q2 + q0);
    return (c0 >= -t0 && c1 >= -t1 && c2 >= -t2) || (c0 <= t0 && c1 <= t1 && c2 <= t2);
}

// atan2 by octant reduction and t*P(t^2) on t in [0, 1]; the coefficients
// are a weighted least-squares fit of atan on [0, 1] made for this file (max
// error of the FP32 evaluation 3.2e-7 rad, plus the reduction's roundings:
// callers pad the result by 2e-6 rad)
constexpr float ATAN_C0 = 0.9999960660934448f, ATAN_C1 = -0.33317309617996216f, ATAN_C2 = 0.19807466864585876f,
                ATAN_C3 = -0.13232387602329254f, ATAN_C4 = 0.07961045205593109f, ATAN_C5 = -0.03359520062804222f,
                ATAN_C6 = 0.006809381302446127f;
constexpr float FAST_ATAN_PAD = 2e-6f;

__device__ __forceinline__ float fast_atan2(float y, float x) {
    float ax = fabsf(x), ay = fabsf(y);
    float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    // (a subnormal mx would be flushed to zero by the division)
    float t = mx >= 1.17549435e-38f ? div_ftz(mn, mx) : 0.f;
    float t2 = t * t;
    float r = fmaf(t2, ATAN_C6, ATAN_C5);
    r = fmaf(t2, r, ATAN_C4);
    r = fmaf(t2, r, ATAN_C3);
    r = fmaf(t2, r, ATAN_C2);
    r = fmaf(t2, r, ATAN_C1);
    r = fmaf(t2, r, ATAN_C0);
    r *= t;
    if (ay > ax) r = 1.5707963f - r;
    if (x < 0.f) r = 3.1415927f - r;
    return copysignf(r, y);
}

// first channel j with sin(elev_j) >= x (lower) / > x (upper), via the table
__device__ __forceinline__ int lut_bin(const SensorDev& S, float x) {
    float fb = (x - S.lut_lo) * S.lut_inv_w;
    return fb <= 0.f ? 0 : (fb >= (float)(LUT_BINS - 1) ? LUT_BINS - 1 : (int)fb);
}
__device__ __forceinline__ float sin_at(const float* t, int j) { return t[j]; }
__device__ __forceinline__ float sin_at(const float2* t, int j) { return t[j].x; }
template <typename T>
__device__ __forceinline__ int chan_lower(const SensorDev& S, const T* ch, const uint16_t* lut, float x) {
    int j = lut[lut_bin(S, x)], n = (int)S.n_ch;
    while (j < n && sin_at(ch, j) < x) ++j;
    return j;
}
template <typename T>
__device__ __forceinline__ int chan_upper(const SensorDev& S, const T* ch, const uint16_t* lut, float x) {
    int j = lut[lut_bin(S, x)], n = (int)S.n_ch;
    while (j < n && sin_at(ch, j) <= x) ++j;
    return j;
}

// Elevation range (sine) of the triangle's directions.  Vertex values, then
// per edge: long edges add their interior great-circle extremum; short edges
// (angular length alpha <= (pi/2)|e|/min(|a|,|b|) < 5e-3) instead widen the
// range by alpha^2/8, the most a great-circle arc of length alpha rises above
// its endpoints.  Returns whether the vertical axis meets the triangle.
__device__ __forceinline__ bool elev_range(const V3 p[3], float& smin, float& smax) {
    float r2[3], sv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r2[k] = p[k].x * p[k].x + p[k].y * p[k].y + p[k].z * p[k].z;
        sv[k] = r2[k] > 0.f ? p[k].z * rsqrtf(r2[k]) : 0.f;
    }
    smin = fminf(sv[0], fminf(sv[1], sv[2]));
    smax = fmaxf(sv[0], fmaxf(sv[1], sv[2]));
    float dev = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int k1 = k == 2 ? 0 : k + 1;
        V3 a = p[k], b = p[k1];
        float ex = b.x - a.x, ey = b.y - a.y, ez = b.z - a.z;
        float ee = ex * ex + ey * ey + ez * ez;
        float m2 = fminf(r2[k], r2[k1]);
        if (ee < 1e-5f * m2)
            dev = fmaxf(dev, 0.31f * ee * __frcp_ru(m2));
        else
            edge_elev_extremum(a, b, smin, smax);
    }
    smin -= dev;
    smax += dev;
    bool pierced = axis_pierces(p);
    if (pierced) {
        if (fmaxf(p[0].z, fmaxf(p[1].z, p[2].z)) > 0.f) smax = 1.f;
        if (fminf(p[0].z, fminf(p[1].z, p[2].z)) < 0.f) smin = -1.f;
    }
    return pierced;
}

// World-frame (rotation-free) elevation range for phase A: only z = u.w and
// |w|^2 per vertex are needed, both invariant under the emitter rotation.
// Same bounds as elev_range; the vertical-axis test runs in the emitter frame
// only when a necessary condition holds: the projected triangle can contain
// the origin only if its nearest vertex lies within the longest edge of it.
__device__ __forceinline__ bool elev_range_w(const SensorDev& S, const V3 w[3], const float eeT[3], float& smin,
                                             float& smax) {
    const V3 u = {S.B[6], S.B[7], S.B[8]};
    float z[3], r2[3], sv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        z[k] = u.x * w[k].x + u.y * w[k].y + u.z * w[k].z;
        r2[k] = w[k].x * w[k].x + w[k].y * w[k].y + w[k].z * w[k].z;
        sv[k] = r2[k] > 0.f ? z[k] * rsqrtf(r2[k]) : 0.f;
    }
    smin = fminf(sv[0], fminf(sv[1], sv[2]));
    smax = fmaxf(sv[0], fmaxf(sv[1], sv[2]));
    const float r2min = fminf(r2[0], fminf(r2[1], r2[2]));
    const float r2max = fmaxf(r2[0], fmaxf(r2[1], r2[2]));
    // upper bound of |w[k1]-w[k]|^2 from the world-frame edge E (sensor
    // independent): |w[k1]-w[k]| <= |E|(1+u) + 4u|w|, so
    // |w[k1]-w[k]|^2 <= 1.0001 |E|^2 + 1.6e5 (4u)^2 |w|^2 / 16; ee_max bounds all three
    const float ee_max = 1.0001f * fmaxf(eeT[0], fmaxf(eeT[1], eeT[2])) + 5.7e-10f * r2max;
    float dev = 0.f;
    if (ee_max < 1e-4f * r2min && r2min > 1e-30f && r2min < 1e36f) {
        // every edge is short (below): one bound for the three,
        // 0.31 ee_max / r2min >= 0.31 ee / m2 of each edge
        dev = 0.3100004f * __fdividef(ee_max, r2min);
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int k1 = k == 2 ? 0 : k + 1;
            V3 a = w[k];
            float m2 = fminf(r2[k], r2[k1]);
            float ee = 1.0001f * eeT[k] + 5.7e-10f * fmaxf(r2[k], r2[k1]);
            if (ee < 1e-4f * m2 && m2 > 1e-30f && m2 < 1e36f) {
                // 0.31 ee / m2 with the fast division (2 ulp) rounded up by the constant;
                // alpha <= 0.016 rad here, where the arc's rise stays below 0.3085 ee / m2
                dev = fmaxf(dev, 0.3100004f * __fdividef(ee, m2));
            } else {
                V3 e = {w[k1].x - a.x, w[k1].y - a.y, w[k1].z - a.z};
                ee = e.x * e.x + e.y * e.y + e.z * e.z;
                // interior extremum of the edge's great circle: +-|m_h|/|m|, m = a x e
                float ez = z[k1] - z[k];
                float ae = a.x * e.x + a.y * e.y + a.z * e.z;
                float num = z[k] * ae - ez * r2[k];
                float den = ez * ae - z[k] * ee;
                if (den < 0.f) {
                    num = -num;
                    den = -den;
                }
                if (den > 0.f && num > -1e-3f * den && num < 1.001f * den) {
                    V3 m = {a.y * e.z - a.z * e.y, a.z * e.x - a.x * e.z, a.x * e.y - a.y * e.x};
                    float mm = m.x * m.x + m.y * m.y + m.z * m.z;
                    float mz = u.x * m.x + u.y * m.y + u.z * m.z;
                    if (mm > 1e-12f * r2[k] * ee) {
                        float v = sqrtf(fmaxf(mm - mz * mz, 0.f) * __frcp_rn(mm));
                        float lam = fminf(fmaxf(num / den, 0.f), 1.f);
                        float qz = z[k] + lam * ez;
                        float tol = 1e-4f * sqrtf(r2[k] + ee);
                        if (qz >= -tol) smax = fmaxf(smax, v);
                        if (qz <= tol) smin = fminf(smin, -v);
                    }
                }
            }
        }
    }
    smin -= dev;
    smax += dev;
    float h2min = fminf(r2[0] - z[0] * z[0], fminf(r2[1] - z[1] * z[1], r2[2] - z[2] * z[2]));
    bool pierced = false;
    if (h2min <= 1.01f * ee_max + 8.f * U32 * r2max) {
        V3 p[3] = {rotB(S.B, w[0]), rotB(S.B, w[1]), rotB(S.B, w[2])};
        pierced = axis_pierces(p);
    }
    if (pierced) {
        if (fmaxf(z[0], fmaxf(z[1], z[2])) > 0.f) smax = 1.f;
        if (fminf(z[0], fminf(z[1], z[2])) < 0.f) smin = -1.f;
    }
    if (!(r2max < 3e38f)) {
        // a vertex so far away that |w|^2 overflows: every channel, full circle
        smin = -1.f;
        smax = 1.f;
        pierced = true;
    }
    return pierced;
}

// azimuth padding of vertex p from |p|^2 and |p_h|^2 (10 rad, the full
// circle, near the vertical axis and where r2 * h2 could overflow)
__device__ __forceinline__ float az_pad2(V3 p) {
    float h2 = p.x * p.x + p.y * p.y;
    float r2 = h2 + p.z * p.z;
    return h2 > 1e-12f * r2 && r2 < 1e18f ? 16.f * U32 * r2 * rsqrt_ftz(r2 * h2) : 10.f;
}

// closest-point distance from the origin to the triangle (w = vertices
// relative to the origin), for the range cull (App. A.4.1 Step 1: delta_min)
__device__ __forceinline__ float closest_dist(V3 a, V3 b, V3 c) {
    V3 ab = {b.x - a.x, b.y - a.y, b.z - a.z}, ac = {c.x - a.x, c.y - a.y, c.z - a.z};
    V3 ap = {-a.x, -a.y, -a.z};
    float d1 = ab.x * ap.x + ab.y * ap.y + ab.z * ap.z, d2 = ac.x * ap.x + ac.y * ap.y + ac.z * ap.z;
    if (d1 <= 0.f && d2 <= 0.f) return sqrtf(a.x * a.x + a.y * a.y + a.z * a.z);
    V3 bp = {-b.x, -b.y, -b.z};
    float d3 = ab.x * bp.x + ab.y * bp.y + ab.z * bp.z, d4 = ac.x * bp.x + ac.y * bp.y + ac.z * bp.z;
    if (d3 >= 0.f && d4 <= d3) return sqrtf(b.x * b.x + b.y * b.y + b.z * b.z);
    float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
        float v = d1 / (d1 - d3);
        V3 q = {a.x + v * ab.x, a.y + v * ab.y, a.z + v * ab.z};
        return sqrtf(q.x * q.x + q.y * q.y + q.z * q.z);
    }
    V3 cp = {-c.x, -c.y, -c.z};
    float d5 = ab.x * cp.x + ab.y * cp.y + ab.z * cp.z, d6 = ac.x * cp.x + ac.y * cp.y + ac.z * cp.z;
    if (d6 >= 0.f && d5 <= d6) return sqrtf(c.x * c.x + c.y * c.y + c.z * c.z);
    float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
        float w = d2 / (d2 - d6);
        V3 q = {a.x + w * ac.x, a.y + w * ac.y, a.z + w * ac.z};
        return sqrtf(q.x * q.x + q.y * q.y + q.z * q.z);
    }
    float va = d3 * d6 - d5 * d4;
    if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
        float w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        V3 q = {b.x + w * (c.x - b.x), b.y + w * (c.y - b.y), b.z + w * (c.z - b.z)};
        return sqrtf(q.x * q.x + q.y * q.y + q.z * q.z);
    }
    float den = 1.f / (va + vb + vc);
    float v = vb * den, w = vc * den;
    V3 q = {a.x + ab.x * v + ac.x * w, a.y + ab.y * v + ac.y * w, a.z + ab.z * v + ac.z * w};
    return sqrtf(q.x * q.x + q.y * q.y + q.z * q.z);
}

// ---------------------------------------------------------------------------
// k_init
// ---------------------------------------------------------------------------
__global__ void k_init(CastArgs a) {
    uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (uint32_t g = tid; g < a.n_rays_total; g += stride) a.keys[g] = KEY_MISS;
    uint32_t nw = (a.n_rays_total + 31u) >> 5;
    for (uint32_t q = tid; q < nw; q += stride) a.flag_bits[q] = 0u;
    if (tid < Q_NUM) a.qcount[tid] = 0u;
    if (tid < C_NUM) a.counters[tid] = 0ull;
    if (tid == 0) *a.error = 0u;
}

// ---------------------------------------------------------------------------
// k_cull: persistent over triangle blocks, all sensors of the cast per triangle
// ---------------------------------------------------------------------------
__device__ __forceinline__ void warp_add(unsigned long long* ctr, uint32_t v) {
    uint32_t s = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, (unsigned long long)s);
}

// ---------------------------------------------------------------------------
// culling, shared by the fused kernel (k_cull) and the split pair (k_cull_a,
// k_cull_b)
// ---------------------------------------------------------------------------
struct CullCounters {
    uint32_t live = 0, cand = 0, inl = 0, big = 0, tests = 0, hits = 0, unc = 0, ties = 0;
    __device__ void flush(const CastArgs& a) const {
        warp_add(&a.counters[C_PAIRS_LIVE], live);
        warp_add(&a.counters[C_CAND], cand);
        warp_add(&a.counters[C_CAND_INLINE], inl);
        warp_add(&a.counters[C_BIG], big);
        warp_add(&a.counters[C_TESTS], tests);
        warp_add(&a.counters[C_HITS], hits);
        warp_add(&a.counters[C_UNCERTAIN], unc);
        warp_add(&a.counters[C_TIES], ties);
    }
};

// channel span bits: j_lo | j_hi << 10 | pierced << 20  (channels < 1024)
__device__ __forceinline__ uint32_t pack_span(int jl, int jh, bool pierced) {
    return (uint32_t)jl | ((uint32_t)jh << 10) | (pierced ? (1u << 20) : 0u);
}

// Phase A of one (triangle, sensor) pair: back-face cull (if requested) and
// the channel span from the elevation range.  Returns false when culled.
template <bool RECHECK, bool BRUTE, typename T>
__device__ __forceinline__ bool cull_elevation(const SensorDev& S, const T* ch, const uint16_t* lut, const V3 v[3],
                                               const V3& nw, const float eeT[3], float lmax, bool cull_back,
                                               bool lossy_area, float area_eps2, uint32_t& span) {
    V3 w0 = rel_origin(S, v[0]);
    if (cull_back) {
        float det = vdot(w0, nw);
        V3 e1 = vsub(v[1], v[0]), e2 = vsub(v[2], v[0]);
        const V3 N = {fabsf(e1.y * e2.z) + fabsf(e1.z * e2.y), fabsf(e1.z * e2.x) + fabsf(e1.x * e2.z),
                      fabsf(e1.x * e2.y) + fabsf(e1.y * e2.x)};
        if (det > 0.f && (!RECHECK || det > backface_err(w0, nw, N))) return false;  // facing <=> det < 0
    }
    if (BRUTE) {
        span = pack_span(0, (int)S.n_ch - 1, false);
        return true;
    }
    const V3 wv[3] = {w0, rel_origin(S, v[1]), rel_origin(S, v[2])};
    if (S.d_max < INFINITY) {
        // range pre-cull (App. A.4.1 Step 1), only where provably empty: every
        // point of the triangle lies within lmax (the longest edge) of vertex 0,
        // so its distance is within |w0| -+ lmax; skipped for unlimited range,
        // where a d_min of centimetres would almost never drop a pair
        const float d0 = sqrtf(vdot(wv[0], wv[0]));
        if (d0 - lmax > S.d_max * (1.f + 2e-5f) + 2e-6f) return false;
        if (d0 + lmax < S.d_min * (1.f - 2e-5f) - 2e-6f) return false;
    }
    if (lossy_area) {
        // Eq. apparent_area: A_T (c-o).n^ = (c-o).n / 2 with n = (v1-v0)x(v2-v0)
        V3 wc = {(wv[0].x + wv[1].x + wv[2].x) * (1.f / 3.f), (wv[0].y + wv[1].y + wv[2].y) * (1.f / 3.f),
                 (wv[0].z + wv[1].z + wv[2].z) * (1.f / 3.f)};
        float dc = 0.5f * (wc.x * nw.x + wc.y * nw.y + wc.z * nw.z);
        float r2c = wc.x * wc.x + wc.y * wc.y + wc.z * wc.z;
        if (dc * dc < area_eps2 * r2c * r2c * r2c) return false;
    }
    float smin, smax;
    bool pierced = elev_range_w(S, wv, eeT, smin, smax);
    int jl = chan_lower(S, ch, lut, smin - EPS_S);
    if (jl >= (int)S.n_ch || sin_at(ch, jl) > smax + EPS_S) return false;  // no channel in the range
    int jh = chan_upper(S, ch, lut, smax + EPS_S) - 1;
    span = pack_span(jl, jh, pierced);
    return true;
}

// Phase B of a surviving pair: range cull, azimuth span, then inline tests or
// a deferred-queue append.
template <bool RECHECK, bool BRUTE>
__device__ __forceinline__ void cull_rest(const CastArgs& a, const SensorDev& S, uint32_t sn, const float2* chs,
                                          uint32_t tri, const float* t9, uint32_t span, CullCounters& c) {
    const bool dump = a.flags & 16u;
    V3 vv[3] = {{t9[0], t9[1], t9[2]}, {t9[3], t9[4], t9[5]}, {t9[6], t9[7], t9[8]}};
    V3 w[3], p[3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
        w[kk] = rel_origin(S, vv[kk]);
        p[kk] = rotB(S.B, w[kk]);
    }
    if (!BRUTE && S.has_range) {
        // range cull (App. A.4.1 Step 1), only where provably empty
        float dmax2 = fmaxf(vdot(w[0], w[0]), fmaxf(vdot(w[1], w[1]), vdot(w[2], w[2])));
        float dlo = fmaxf(S.d_min * (1.f - 1e-5f) - 1e-6f, 0.f);
        if (dmax2 < dlo * dlo) return;
        if (S.d_max < INFINITY && closest_dist(w[0], w[1], w[2]) > S.d_max * (1.f + 1e-5f) + 1e-6f) return;
    }
    Span sp;
    sp.j_lo = (int)(span & 1023u);
    sp.j_hi = (int)((span >> 10) & 1023u);
    sp.pierced = (span >> 20) & 1u;
    if (BRUTE) {
        sp.u_lo = 0;
        sp.n_r = (int)S.n_rays;
        sp.a0 = 0.f;
    } else {
        sp.a0 = ray_units(S, fast_atan2(p[0].y, p[0].x));
        float A, B;
        if (sp.pierced) {
            A = sp.a0 - 0.5f * S.period;
            B = sp.a0 + 0.5f * S.period;
        } else {
            float d1 = rel_angle(p[0], p[1]);
            float d2 = rel_angle(p[0], p[2]);
            float pad = EPS_T + 3.f * FAST_ATAN_PAD + az_pad2(p[0]) + az_pad2(p[1]) + az_pad2(p[2]);
            float lo = fminf(0.f, fminf(d1, d2)) - pad, hi = fmaxf(0.f, fmaxf(d1, d2)) + pad;
            if (hi - lo >= 6.2831f) {
                A = sp.a0 - 0.5f * S.period;
                B = sp.a0 + 0.5f * S.period;
            } else {
                A = sp.a0 + lo * S.inv_dtheta;
                B = sp.a0 + hi * S.inv_dtheta;
            }
        }
        if (!ray_interval(S, A - PADR - S.az_noise_pad, B + PADR + S.az_noise_pad, sp.u_lo, sp.n_r)) return;
    }
    const uint32_t ncand = (uint32_t)(sp.j_hi - sp.j_lo + 1) * (uint32_t)sp.n_r;
    c.live++;
    c.cand += ncand;
    if (!BRUTE && ncand > a.inline_max) {
        // deferred list append: one atomic per coalesced group (ballot + popc rank)
        cg::coalesced_group grp = cg::coalesced_threads();
        uint32_t b0 = 0;
        if (grp.thread_rank() == 0) b0 = atomicAdd(&a.qcount[Q_BIG], grp.size());
        b0 = grp.shfl(b0, 0) + grp.thread_rank();
        if (b0 < a.big_cap) {
            BigPair bp;
            bp.tri = tri;
            bp.sensor = (uint16_t)sn;
            bp.flags = sp.pierced ? 1 : 0;
            bp.j_lo = (uint16_t)sp.j_lo;
            bp.j_hi = (uint16_t)sp.j_hi;
            bp.u_lo = sp.u_lo;
            bp.n_r = (uint32_t)sp.n_r;
            bp.a0 = sp.a0;
            bp.pad_[0] = bp.pad_[1] = 0;
            a.big[b0] = bp;
        } else {
            atomicOr(a.error, (uint32_t)ERR_BIG_CAP);
        }
        c.big++;
        return;
    }
    TriW T;
    tri_world(t9, T);
    float det = vdot(w[0], T.n);
    float err_det = det_error(w[0], T);
    bool det_unc = fabsf(det) <= err_det;
    if (det == 0.f && !(RECHECK && det_unc)) return;  // origin in the plane: t = 0, never a hit
    c.inl += ncand;
    PairSetup st;
    make_setup(S, T, w, p, det, err_det, SetupWriterAoS{st});
    const float2* azs = a.az_sc + S.az_off;
    const int n = (int)S.n_rays;
    const int r0 = imod(sp.u_lo, n);
    for (int j = sp.j_lo; j <= sp.j_hi; ++j) {
        const float2 chv = chs[j];
        const uint32_t gbase = S.ray_off + (uint32_t)j * (uint32_t)n;
        int i = r0;
        for (int qq = 0; qq < sp.n_r; ++qq) {
            V3 d = ray_dir(chv, __ldg(&azs[i]));
            float t, terr;
            int res = test_fp32<RECHECK>(SetupAoS{st}, S, d, t, terr);
            c.tests++;
            if (dump) dump_candidate(a, gbase + i, tri);
            c.hits += commit<RECHECK>(a, gbase + i, tri, res, t, terr, st.t_lb, c.unc, c.ties);
            if (++i == n) i = 0;
        }
    }
}

// shared-memory prologue: sensor descriptors, channel tables, lookup tables
struct CullSmem {
    SensorDev* sens;
    float2* ch;
    uint16_t* lut;
    unsigned char* rest;  // 16-B aligned
};
__device__ __forceinline__ CullSmem cull_smem_prologue(const CastArgs& a, unsigned char* smem, bool with_lut) {
    CullSmem m;
    m.sens = reinterpret_cast<SensorDev*>(smem);
    m.ch = reinterpret_cast<float2*>(smem + sizeof(SensorDev) * a.n_sensors);
    m.lut = reinterpret_cast<uint16_t*>(smem + sizeof(SensorDev) * a.n_sensors + sizeof(float2) * a.total_ch);
    size_t off = sizeof(SensorDev) * a.n_sensors + sizeof(float2) * a.total_ch +
                 (with_lut ? sizeof(uint16_t) * LUT_BINS * a.n_sensors : 0);
    off = (off + 15) & ~size_t(15);
    m.rest = smem + off;
    for (uint32_t q = threadIdx.x; q < a.n_sensors * (uint32_t)(sizeof(SensorDev) / 4); q += blockDim.x)
        reinterpret_cast<uint32_t*>(m.sens)[q] = reinterpret_cast<const uint32_t*>(a.sensors)[q];
    __syncthreads();
    for (uint32_t sn = 0; sn < a.n_sensors; ++sn) {
        const SensorDev& S = m.sens[sn];
        for (uint32_t j = threadIdx.x; j < S.n_ch; j += blockDim.x) m.ch[S.ch_loc + j] = a.ch_sc[S.ch_off + j];
        if (with_lut)
            for (uint32_t b = threadIdx.x; b < LUT_BINS; b += blockDim.x) m.lut[sn * LUT_BINS + b] = a.lut[S.lut_off + b];
    }
    __syncthreads();
    return m;
}

// stage a warp's 32 triangles (1152 B, 16-B aligned since base % 4 == 0)
__device__ __forceinline__ void stage_tris(const CastArgs& a, uint32_t base, uint32_t cnt, float* dst, uint32_t lane) {
    const float4* src = reinterpret_cast<const float4*>(a.tris + 9ull * base);
    const uint32_t n4 = (cnt * 9u + 3u) >> 2;
    __syncwarp();
    for (uint32_t q = lane; q < n4; q += 32) reinterpret_cast<float4*>(dst)[q] = __ldcs(src + q);
    __syncwarp();
}

// Same for a caller-owned buffer that ends right after triangle n_tris - 1
// (no tail padding): whole float4s up to the buffer's end, the last 1-3
// floats of an odd-sized tail by scalar loads.
__device__ __forceinline__ void stage_tris_bounded(const CastArgs& a, uint32_t base, uint32_t cnt, float* dst,
                                                   uint32_t lane) {
    const float* src = a.tris + 9ull * base;
    const uint32_t nf = cnt * 9u, n4 = nf >> 2;
    __syncwarp();
    for (uint32_t q = lane; q < n4; q += 32)
        reinterpret_cast<float4*>(dst)[q] = __ldcs(reinterpret_cast<const float4*>(src) + q);
    if (lane < (nf & 3u)) dst[4 * n4 + lane] = __ldcs(src + 4 * n4 + lane);
    __syncwarp();
}

// ---------------------------------------------------------------------------
// k_cull (fused): phase A, warp compaction of the survivors, phase B
// ---------------------------------------------------------------------------
constexpr int CULL_GROUP = 8;  // sensors per elevation phase
struct CullWarpSmem {
    float tri[32 * 9 + 4];            // staged triangles (+ one float4 of slack)
    uint32_t span[32 * CULL_GROUP];   // channel span per (lane, sensor)
    uint16_t list[32 * CULL_GROUP];   // surviving (lane, sensor) pairs: lane | k << 5
};
static_assert(sizeof(CullWarpSmem) % 16 == 0, "per-warp staging must stay 16-byte aligned");

template <bool RECHECK, bool BRUTE>
__global__ void __launch_bounds__(256, 3) k_cull(CastArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    CullSmem M = cull_smem_prologue(a, smem, true);
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    CullWarpSmem& W = reinterpret_cast<CullWarpSmem*>(M.rest)[wib];
    const bool cull_back = a.flags & 2u;
    CullCounters c;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t gwarp = ((blockIdx.x * blockDim.x) >> 5) + wib;
    for (uint32_t base = gwarp * 32; base < a.n_tris; base += n_warps * 32) {
        const uint32_t cnt = min(32u, a.n_tris - base);
        stage_tris_bounded(a, base, cnt, W.tri, lane);
        bool valid = lane < cnt;
        const float* t9 = W.tri + 9 * (valid ? lane : 0);
        V3 v[3] = {{t9[0], t9[1], t9[2]}, {t9[3], t9[4], t9[5]}, {t9[6], t9[7], t9[8]}};
        V3 nw = vcross(vsub(v[1], v[0]), vsub(v[2], v[0]));
        if (nw.x == 0.f && nw.y == 0.f && nw.z == 0.f) valid = false;  // zero area: never hit
        float eeT[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            V3 e = vsub(v[k == 2 ? 0 : k + 1], v[k]);
            eeT[k] = vdot(e, e);
        }
        // longest edge, rounded up (sensor independent)
        const float lmax = sqrtf(fmaxf(eeT[0], fmaxf(eeT[1], eeT[2]))) * (1.f + 1e-6f);
        for (uint32_t sg = 0; sg < a.n_sensors; sg += CULL_GROUP) {
            const uint32_t ng = min((uint32_t)CULL_GROUP, a.n_sensors - sg);
            uint32_t mask = 0;
            if (valid) {
                for (uint32_t k = 0; k < ng; ++k) {
                    uint32_t span;
                    if (cull_elevation<RECHECK, BRUTE>(M.sens[sg + k], M.ch + M.sens[sg + k].ch_loc,
                                                       M.lut + (sg + k) * LUT_BINS, v, nw, eeT, lmax, cull_back,
                                                       (a.flags & 32u) != 0, a.area_eps2, span)) {
                        mask |= 1u << k;
                        W.span[lane * CULL_GROUP + k] = span;
                    }
                }
            }
            const uint32_t my = __popc(mask);
            uint32_t incl = my;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += t;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            {
                uint32_t at = incl - my, m = mask;
                while (m) {
                    uint32_t k = __ffs(m) - 1;
                    m &= m - 1;
                    W.list[at++] = (uint16_t)(lane | (k << 5));
                }
            }
            __syncwarp();
            for (uint32_t q0 = 0; q0 < total; q0 += 32) {
                const uint32_t q = q0 + lane;
                if (q < total) {
                    const uint32_t e = W.list[q];
                    const uint32_t srcl = e & 31u, k = e >> 5, sn = sg + k;
                    cull_rest<RECHECK, BRUTE>(a, M.sens[sn], sn, M.ch + M.sens[sn].ch_loc, base + srcl,
                                              W.tri + 9 * srcl, W.span[srcl * CULL_GROUP + k], c);
                }
            }
            __syncwarp();
        }
    }
    c.flush(a);
}

// ---------------------------------------------------------------------------
// k_cull_a: phase A over all pairs; survivors go to a global queue through a
// per-warp shared-memory buffer (one atomic per flush of >= 256 entries)
// record: tri | span << 32 | sensor << 53
// ---------------------------------------------------------------------------
constexpr int ELEV_GROUP = 8;  // sensors per k_cull_a launch (the sensor loop is unrolled over them)
constexpr int SURV_BUF = 352;    // per-warp survivor buffer; flushed before a step could overflow it
struct CullAWarpSmem {
    float tri[32 * 9 + 4];
    unsigned long long buf[SURV_BUF];
};
static_assert(sizeof(CullAWarpSmem) % 16 == 0, "per-warp staging must stay 16-byte aligned");
static_assert(SURV_BUF >= 32 * ELEV_GROUP, "a tile must fit an empty buffer");

// Flush a warp's survivor buffer to the global queue in its order: one
// atomic for the whole buffer, coalesced 8-byte stores.  The sensor loop
// appends a tile's survivors sensor by sensor, so a batch of 32 survivors in
// k_cull_b holds runs of a few sensors.  (A counting sort by sensor here, to
// give k_cull_b single-sensor batches, cost k_cull_a 15 % and saved k_cull_b
// nothing.)
__device__ __forceinline__ void flush_survivors(const CastArgs& a, CullAWarpSmem& W, uint32_t& fill, uint32_t lane) {
    if (fill == 0) return;
    uint32_t b0 = 0;
    if (lane == 0) b0 = atomicAdd(&a.qcount[Q_SURV], fill);
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    for (uint32_t q = lane; q < fill; q += 32) {
        const uint32_t dst = b0 + q;
        if (dst < a.surv_cap)
            a.surv[dst] = W.buf[q];
        else
            atomicOr(a.error, (uint32_t)ERR_SURV_CAP);
    }
    __syncwarp();
    fill = 0;
}

// ---------------------------------------------------------------------------
// GACP-T_g (Sec. 10.1.1): the emitter test lifted from one triangle to the
// bounding box of a 32-triangle group.  A group is dropped for a sensor when
// the box lies wholly beyond the range limits or when the elevation range of
// its bounding sphere, seen from the sensor, holds no channel.  Every member's
// own (padded) elevation range lies inside the sphere's, so the group test
// never drops a pair that the per-triangle cull would keep.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool group_may_hit(const SensorDev& S, const float* sins, const uint16_t* lut,
                                              const float4& lo, const float4& hi) {
    // a box with an infinite side (a member with an infinite vertex) bounds
    // nothing useful: keep the group
    if (!isfinite(lo.x + lo.y + lo.z + hi.x + hi.y + hi.z)) return true;
    // rounding of w = (v - o_hi) - o_lo is monotone in v, so every member
    // vertex, transformed like the triangles, lies inside [wl, wh]
    const V3 wl = rel_origin(S, V3{lo.x, lo.y, lo.z}), wh = rel_origin(S, V3{hi.x, hi.y, hi.z});
    if (S.has_range) {
        const float nx = fmaxf(fmaxf(wl.x, -wh.x), 0.f), ny = fmaxf(fmaxf(wl.y, -wh.y), 0.f),
                    nz = fmaxf(fmaxf(wl.z, -wh.z), 0.f);
        const float dmax = S.d_max * (1.f + 3e-5f) + 3e-6f;  // d_max may be +inf
        if (nx * nx + ny * ny + nz * nz > dmax * dmax) return false;
        const float fx = fmaxf(fabsf(wl.x), fabsf(wh.x)), fy = fmaxf(fabsf(wl.y), fabsf(wh.y)),
                    fz = fmaxf(fabsf(wl.z), fabsf(wh.z));
        const float dmin = fmaxf(S.d_min * (1.f - 3e-5f) - 3e-6f, 0.f);
        if (fx * fx + fy * fy + fz * fz < dmin * dmin) return false;
    }
    const V3 c = {0.5f * (wl.x + wh.x), 0.5f * (wl.y + wh.y), 0.5f * (wl.z + wh.z)};
    const V3 h = {0.5f * (wh.x - wl.x), 0.5f * (wh.y - wl.y), 0.5f * (wh.z - wl.z)};
    const float R = sqrtf(vdot(h, h)) * (1.f + 1e-6f) + 2e-7f * (fabsf(c.x) + fabsf(c.y) + fabsf(c.z));
    const float D2 = vdot(c, c);
    // near or large spheres (half-angle above ~82 deg): keep, the bound is loose there
    if (!(D2 > 0.f) || !(D2 < 3e38f) || R * R > 0.98f * D2) return true;
    const float invD = rsqrtf(D2);
    // centre elevation from the sensor frame (no cancellation near the poles)
    const float cx = S.B[0] * c.x + S.B[1] * c.y + S.B[2] * c.z, cy = S.B[3] * c.x + S.B[4] * c.y + S.B[5] * c.z,
                cz = S.B[6] * c.x + S.B[7] * c.y + S.B[8] * c.z;
    const float sphi = fminf(fmaxf(cz * invD, -1.f), 1.f);
    const float cphi = fminf(sqrtf(cx * cx + cy * cy) * invD, 1.f);
    const float sa = R * invD, ca = sqrtf(fmaxf(1.f - sa * sa, 0.f));
    // elevation range of the cap of half-angle alpha around the centre direction
    const float shi = (cphi * ca - sphi * sa < 0.f) ? 1.f : sphi * ca + cphi * sa;
    const float slo = (cphi * ca + sphi * sa < 0.f) ? -1.f : sphi * ca - cphi * sa;
    constexpr float PAD = 3e-5f;  // > FP32 error of this bound + the per-triangle padding
    const int jl = chan_lower(S, sins, lut, slo - PAD);
    return jl < (int)S.n_ch && sin_at(sins, jl) <= shi + PAD;
}

// one warp per 32-triangle group: box of its (present) vertices
__global__ void k_group_bounds(const float* __restrict__ tris, uint32_t n_tris, uint32_t g0, uint32_t g1,
                               float4* __restrict__ gb) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t g = g0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); g < g1; g += n_warps) {
        const uint32_t t = g * GROUP_TRIS + lane;
        float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
        if (t < n_tris) {
            const float* v = tris + 9ull * t;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float x = __ldg(v + 3 * k), y = __ldg(v + 3 * k + 1), z = __ldg(v + 3 * k + 2);
                lx = fminf(lx, x);
                ly = fminf(ly, y);
                lz = fminf(lz, z);
                hx = fmaxf(hx, x);
                hy = fmaxf(hy, y);
                hz = fmaxf(hz, z);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
            ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
            lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
            hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
            hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
            hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        }
        if (lane == 0) {
            gb[2ull * g] = make_float4(lx, ly, lz, 0.f);
            gb[2ull * g + 1] = make_float4(hx, hy, hz, 0.f);
        }
    }
}

void launch_group_bounds(const float* tris, uint32_t n_tris, uint32_t first, uint32_t n, float4* gb, int n_sm,
                         cudaStream_t st) {
    if (n == 0 || n_tris == 0) return;
    const uint32_t g0 = first / GROUP_TRIS, g1 = (uint32_t)(((uint64_t)first + n + GROUP_TRIS - 1) / GROUP_TRIS);
    const uint32_t warps = g1 - g0;
    const uint32_t blocks = std::min<uint32_t>((warps + 7) / 8, (uint32_t)n_sm * 8u);
    k_group_bounds<<<std::max(blocks, 1u), 256, 0, st>>>(tris, n_tris, g0, g1, gb);
}

// Per-sensor constants of the elevation pass, four float4 in shared memory
// (one LDS.128 each per sensor step).  The origin's low part o_lo is not
// subtracted per vertex: vertices are taken relative to o_hi and every bound
// that uses them is widened by |o_lo| (olo = 1.01 |o_lo|).
struct __align__(16) ElevSensor {
    float ox, oy, oz, olo;       // o_hi; widening for the origin's low part
    float ux, uy, uz, thr0;      // up axis (row u of B); pierce pre-test constant 101 olo^2 (rounded up)
    float nlo_w, inv_w, dmax, dmin;  // LUT bin = round(s * inv_w + nlo_w); range pre-cull bounds (dmax inf: none)
    uint32_t n_ch, sins_off, lut_off, up;   // up: 1 when the up axis is exactly (0, 0, 1)
};
static_assert(sizeof(ElevSensor) == 64, "four float4");

// prologue of k_cull_a: the launch's sensors (full descriptors for the rare
// paths and the group cull, packed elevation records), channel sines, lookup tables
struct CullASmem {
    SensorDev* sens;
    ElevSensor* es;
    float* sins;
    uint16_t* lut;
    unsigned char* rest;
};
// Layout: the 16-byte ElevSensor records first (read as float4), then the
// SensorDev copies (8-byte aligned after them), the sines and the tables.
static_assert(sizeof(ElevSensor) % 16 == 0 && sizeof(SensorDev) % alignof(SensorDev) == 0 &&
                  alignof(SensorDev) <= 16,
              "k_cull_a shared-memory layout");
__device__ __forceinline__ size_t cull_a_head_bytes(uint32_t ns, uint32_t n_ch) {
    const size_t off = sizeof(ElevSensor) * ns + sizeof(SensorDev) * ns + sizeof(float) * n_ch +
                       sizeof(uint16_t) * LUT_BINS * ns;
    return (off + 15) & ~size_t(15);
}
__device__ __forceinline__ CullASmem cull_a_prologue(const CastArgs& a, unsigned char* smem) {
    CullASmem m;
    const uint32_t ns = a.sens_count, s0 = a.sens_base;
    m.es = reinterpret_cast<ElevSensor*>(smem);
    m.sens = reinterpret_cast<SensorDev*>(smem + sizeof(ElevSensor) * ns);
    m.sins = reinterpret_cast<float*>(smem + (sizeof(SensorDev) + sizeof(ElevSensor)) * ns);
    // the sines of the launch's sensors take at most total_ch entries
    m.lut = reinterpret_cast<uint16_t*>(smem + (sizeof(SensorDev) + sizeof(ElevSensor)) * ns + sizeof(float) * a.total_ch);
    m.rest = smem + cull_a_head_bytes(ns, a.total_ch);
    for (uint32_t q = threadIdx.x; q < ns * (uint32_t)(sizeof(SensorDev) / 4); q += blockDim.x)
        reinterpret_cast<uint32_t*>(m.sens)[q] = reinterpret_cast<const uint32_t*>(a.sensors + s0)[q];
    __syncthreads();
    uint32_t ch_at = 0;
    for (uint32_t k = 0; k < ns; ++k) {
        const SensorDev& S = m.sens[k];
        for (uint32_t j = threadIdx.x; j < S.n_ch; j += blockDim.x) m.sins[ch_at + j] = a.ch_sc[S.ch_off + j].x;
        for (uint32_t b = threadIdx.x; b < LUT_BINS; b += blockDim.x) m.lut[k * LUT_BINS + b] = a.lut[S.lut_off + b];
        if (threadIdx.x == 0) {
            ElevSensor E;
            E.ox = S.o_hi[0];
            E.oy = S.o_hi[1];
            E.oz = S.o_hi[2];
            const float olo = sqrtf(S.o_lo[0] * S.o_lo[0] + S.o_lo[1] * S.o_lo[1] + S.o_lo[2] * S.o_lo[2]);
            E.olo = 1.01f * olo;
            E.ux = S.B[6];
            E.uy = S.B[7];
            E.uz = S.B[8];
            E.thr0 = 101.1f * E.olo * E.olo;
            E.inv_w = S.lut_inv_w;
            E.nlo_w = -S.lut_lo * S.lut_inv_w - 0.25f;
            E.dmax = S.d_max < INFINITY ? S.d_max * (1.f + 2e-5f) + 2e-6f + E.olo : INFINITY;
            E.dmin = S.d_min * (1.f - 2e-5f) - 2e-6f - E.olo;
            E.n_ch = S.n_ch;
            E.sins_off = ch_at;
            E.lut_off = k * LUT_BINS;
            E.up = S.B[6] == 0.f && S.B[7] == 0.f && S.B[8] == 1.f ? 1u : 0u;
            m.es[k] = E;
        }
        ch_at += S.n_ch;
    }
    __syncthreads();
    return m;
}

// first channel whose sine is >= x: lookup-table bin, then a short forward
// scan.  The bin is round(fb - 1/4) (nlo_w holds the -1/4), taken with one
// addition of 1.5 * 2^23, so the bin's start lies at least a quarter bin
// below x: within the table's half-bin slack, with room for rounding.
__device__ __forceinline__ int chan_first(const ElevSensor& E, const float* sins, const uint16_t* lut, float x) {
    const float fb = fminf(fmaxf(fmaf(x, E.inv_w, E.nlo_w), 0.f), (float)(LUT_BINS - 1));
    const uint32_t bin = __float_as_uint(fb + 12582912.f) & 0x3FFFFFu;   // round(fb), 0 <= fb < 2^22
    int j = lut[bin];
    const int n = (int)E.n_ch;
    while (j < n && sins[j] < x) ++j;
    return j;
}

// Phase A of one (triangle, sensor) pair: back-face cull (if requested), the
// range pre-cull, and the channel span from the elevation range.  Returns
// false when culled.  Elevation range (sine space): vertex values, widened by
// dev = 0.31 ee_max / r2min, which bounds how far any edge's great-circle arc
// rises above (or dips below) its endpoints: an arc of angular length alpha
// deviates by at most 1 - cos(alpha / 2) <= alpha^2 / 8 from its higher
// endpoint, and alpha <= (pi / 2) |e| / min(|a|, |b|), so alpha^2 / 8 <=
// (pi^2 / 32) ee / m2 < 0.3085 ee / m2 for every edge; plus |o_lo| / r_min
// for the origin's low part and the FP32 padding EPS_S.  When the vertical
// axis may meet the triangle, the exact test decides and the range opens to
// the pole(s).
// the rare paths of cull_elev, out of line to keep the hot loop small
// back-face cull with the exact origin offset: false when culled
__device__ __noinline__ bool elev_facing(const SensorDev& S, V3 v0, V3 v1, V3 v2, uint32_t flags) {
    const V3 w0 = rel_origin(S, v0);
    const V3 e1 = vsub(v1, v0), e2 = vsub(v2, v0);
    const V3 nw = vcross(e1, e2);
    const float det = vdot(w0, nw);
    if (det > 0.f) {
        if (!(flags & 1u)) return false;
        const V3 N = {fabsf(e1.y * e2.z) + fabsf(e1.z * e2.y), fabsf(e1.z * e2.x) + fabsf(e1.x * e2.z),
                      fabsf(e1.x * e2.y) + fabsf(e1.y * e2.x)};
        if (det > backface_err(w0, nw, N)) return false;  // facing <=> det < 0
    }
    return true;
}
// Eq. apparent_area with the exact origin offset, A_T (c-o).n^ = (c-o).n / 2: false when culled
__device__ __noinline__ bool elev_area_keep(const SensorDev& S, V3 v0, V3 v1, V3 v2, float area_eps2) {
    const V3 wv[3] = {rel_origin(S, v0), rel_origin(S, v1), rel_origin(S, v2)};
    const V3 nw = vcross(vsub(v1, v0), vsub(v2, v0));
    V3 wc = {(wv[0].x + wv[1].x + wv[2].x) * (1.f / 3.f), (wv[0].y + wv[1].y + wv[2].y) * (1.f / 3.f),
             (wv[0].z + wv[1].z + wv[2].z) * (1.f / 3.f)};
    float dc = 0.5f * (wc.x * nw.x + wc.y * nw.y + wc.z * nw.z);
    float r2c = wc.x * wc.x + wc.y * wc.y + wc.z * wc.z;
    return !(dc * dc < area_eps2 * r2c * r2c * r2c);
}
// exact vertical-axis test: bit 0 pierced, bit 1 open to +1, bit 2 open to -1
__device__ __noinline__ uint32_t elev_pierce(const SensorDev& S, V3 v0, V3 v1, V3 v2) {
    const V3 p[3] = {rotB(S.B, rel_origin(S, v0)), rotB(S.B, rel_origin(S, v1)), rotB(S.B, rel_origin(S, v2))};
    if (!axis_pierces(p)) return 0u;
    return 1u | (fmaxf(p[0].z, fmaxf(p[1].z, p[2].z)) > 0.f ? 2u : 0u) |
           (fminf(p[0].z, fminf(p[1].z, p[2].z)) < 0.f ? 4u : 0u);
}

__device__ __forceinline__ bool cull_elev(const ElevSensor& E, const SensorDev& S, const float* sins, const uint16_t* lut,
                                          const V3 v[3], float ee_max, float lmax, uint32_t flags, float area_eps2,
                                          uint32_t& span) {
    if ((flags & 2u) && !elev_facing(S, v[0], v[1], v[2], flags)) return false;
    if (flags & 4u) {  // no culling (debug)
        span = pack_span(0, (int)S.n_ch - 1, false);
        return true;
    }
    float z[3], r2[3], h2[3];
    if (E.up) {  // warp-uniform: an upright sensor needs no projection on u
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float wx = v[k].x - E.ox, wy = v[k].y - E.oy, wz = v[k].z - E.oz;
            z[k] = wz;
            h2[k] = fmaf(wy, wy, wx * wx);
            r2[k] = fmaf(wz, wz, h2[k]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float wx = v[k].x - E.ox, wy = v[k].y - E.oy, wz = v[k].z - E.oz;
            z[k] = fmaf(E.uz, wz, fmaf(E.uy, wy, E.ux * wx));
            r2[k] = fmaf(wz, wz, fmaf(wy, wy, wx * wx));
            h2[k] = fmaf(-z[k], z[k], r2[k]);
        }
    }
    if (E.dmax < INFINITY) {
        // range pre-cull (App. A.4.1 Step 1), only where provably empty: every
        // point of the triangle lies within lmax (the longest edge) of vertex 0
        // (the approximate root's 2^-22 relative error is inside the bounds' padding)
        const float d0 = sqrt_ftz(r2[0]);
        if (d0 - lmax > E.dmax || d0 + lmax < E.dmin) return false;
    }
    if ((flags & 32u) && !elev_area_keep(S, v[0], v[1], v[2], area_eps2)) return false;
    // a vertex at (or within 1e-8 of) the origin can give inf or 0 * inf =
    // NaN here; such a triangle takes the full range below (r2min < 1e-16)
    const float sv0 = z[0] * rsqrt_ftz(r2[0]), sv1 = z[1] * rsqrt_ftz(r2[1]), sv2 = z[2] * rsqrt_ftz(r2[2]);
    const float smin = fminf(sv0, fminf(sv1, sv2)), smax = fmaxf(sv0, fmaxf(sv1, sv2));
    const float r2min = fminf(r2[0], fminf(r2[1], r2[2]));
    const float r2max = fmaxf(r2[0], fmaxf(r2[1], r2[2]));
    const float h2min = fminf(h2[0], fminf(h2[1], h2[2]));
    const float rinv = rsqrt_ftz(fmaxf(r2min, 1e-37f));
    // |w[k1]-w[k]|^2 <= 1.0001 |E|^2 + 5.7e-10 |w|^2 for the FP32 rounding of w
    const float ee_p = fmaf(5.7e-10f, r2max, 1.0001f * ee_max);
    const float dev = fmaf(0.3100004f * ee_p, rinv * rinv, fmaf(E.olo, rinv, EPS_S));
    // (smin, smax are NaN only when every vertex sits at the origin: zero area,
    // never tested; a non-finite vertex takes the overflow branch below)
    float lo = smin - dev, hi = smax + dev;
    bool pierced = false;
    // The vertical axis can meet the projected triangle only if its nearest
    // vertex lies within the longest edge of the axis (with margins for the
    // FP32 rounding and for o_lo: (h + d)^2 <= 1.01 h^2 + 101 d^2).  A vertex
    // so far away that |w|^2 overflows, or within 1e-8 of the origin (it
    // enters the branch since h2min <= r2min), opens every channel and the
    // full circle: near the origin |w|^2 may be subnormal (the flush-to-zero
    // root above then returns +inf), and the per-channel crossings of a
    // deferred pair (k_expand) take products of four coordinates, which
    // underflow below about 1e-9.5.
    if (!(h2min > fmaxf(fmaf(8.2f * U32, r2max, fmaf(1.0201f, ee_max, E.thr0)), 1e-16f)) || !(r2max < 3e38f)) {
        if (!(r2max < 3e38f) || !(r2min >= 1e-16f)) {
            lo = -2.f;
            hi = 2.f;
            pierced = true;
        } else {
            const uint32_t pc = elev_pierce(S, v[0], v[1], v[2]);
            pierced = pc & 1u;
            if (pc & 2u) hi = 2.f;
            if (pc & 4u) lo = -2.f;
        }
    }
    const int n = (int)E.n_ch;
    const int jl = chan_first(E, sins, lut, lo);
    if (jl >= n) return false;
    float sj = sins[jl];
    if (sj > hi) return false;  // no channel in the range
    int jh = jl;
    while (jh + 1 < n) {
        sj = sins[jh + 1];
        if (sj > hi) break;
        ++jh;
    }
    span = pack_span(jl, jh, pierced);
    return true;
}

// k_cull_a: phase A for the sensors [sens_base, sens_base + sens_count) of
// the cast (at most ELEV_GROUP; larger casts launch once per group).  A warp
// stages 32 triangles, keeps their sensor-independent terms in registers and
// runs the unrolled sensor loop over them; survivors go through the warp's
// shared-memory buffer to the global queue.
template <bool GROUPS>
__global__ void __launch_bounds__(256, 4) k_cull_a(CastArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    CullASmem M = cull_a_prologue(a, smem);
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    CullAWarpSmem& W = reinterpret_cast<CullAWarpSmem*>(M.rest)[wib];
    const uint32_t flags = a.flags;
    const uint32_t ns = a.sens_count, s0 = a.sens_base;
    uint32_t fill = 0;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t gwarp = ((blockIdx.x * blockDim.x) >> 5) + wib;
    const bool groups = GROUPS && !(flags & 4u);
    uint32_t g_culled = 0;
    // triangles [0, tri_first) belong to the static hierarchy in a hybrid cast
    const uint32_t first = a.tri_first, base0 = first & ~31u;
    for (uint32_t base = base0 + gwarp * 32; base < a.n_tris; base += n_warps * 32) {
        const uint32_t cnt = min(32u, a.n_tris - base);
        const uint32_t skip = first > base ? first - base : 0u;  // leading lanes outside the range
        uint32_t live = 0xFFu;
        if (groups) {
            // GACP-T_g: lane k tests sensor k against the group's box
            const float4 lo = __ldg(&a.gbounds[2u * (base / GROUP_TRIS)]);
            const float4 hi = __ldg(&a.gbounds[2u * (base / GROUP_TRIS) + 1u]);
            const bool ok = lane < ns && group_may_hit(M.sens[lane], M.sins + M.es[min(lane, ns - 1)].sins_off,
                                                       M.lut + min(lane, ns - 1) * LUT_BINS, lo, hi);
            live = __ballot_sync(0xffffffffu, ok);
            g_culled += (ns - (uint32_t)__popc(live)) * (cnt - skip);
            if (g_culled >= 0x40000000u && lane == 0) {
                atomicAdd(&a.counters[C_GROUP], (unsigned long long)g_culled);
                g_culled = 0;
            }
            if (live == 0) continue;  // the whole tile: no load, no per-triangle work
        }
        if (fill + 32 * ns > SURV_BUF) flush_survivors(a, W, fill, lane);
        stage_tris(a, base, cnt, W.tri, lane);
        {
            // the warp's next tile into L2 while this one is worked on (9 lines of 128 B)
            const uint32_t nb = base + n_warps * 32;
            if (nb < a.n_tris && lane < 9 && 32u * lane < 9u * min(32u, a.n_tris - nb)) {
                const float* pp = a.tris + 9ull * nb + 32 * lane;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(pp));
            }
        }
        bool valid = lane < cnt && lane >= skip;
        const float* t9 = W.tri + 9 * (valid ? lane : 0);
        const V3 v[3] = {{t9[0], t9[1], t9[2]}, {t9[3], t9[4], t9[5]}, {t9[6], t9[7], t9[8]}};
        const V3 e0 = vsub(v[1], v[0]), e1 = vsub(v[2], v[1]), e2 = vsub(v[0], v[2]);
        const V3 nw = vcross(e0, vneg(e2));
        if (nw.x == 0.f && nw.y == 0.f && nw.z == 0.f) valid = false;  // zero area: never hit
        // longest edge (squared; and rounded-up length), sensor independent
        const float ee_max = fmaxf(vdot(e0, e0), fmaxf(vdot(e1, e1), vdot(e2, e2)));
        const float lmax = sqrt_ftz(ee_max) * (1.f + 1e-6f);
#pragma unroll 1
        for (uint32_t k = 0; k < ns; ++k) {
            if (!((live >> k) & 1u)) continue;  // warp-uniform
            uint32_t span = 0;
            const bool ok = valid && cull_elev(M.es[k], M.sens[k], M.sins + M.es[k].sins_off, M.lut + k * LUT_BINS, v,
                                                  ee_max, lmax, flags, a.area_eps2, span);
            const uint32_t bal = __ballot_sync(0xffffffffu, ok);
            if (ok)
                W.buf[fill + __popc(bal & ((1u << lane) - 1u))] = (unsigned long long)(base + lane) |
                                                                   ((unsigned long long)span << 32) |
                                                                   ((unsigned long long)(s0 + k) << 53);
            fill += __popc(bal);
        }
        __syncwarp();
    }
    flush_survivors(a, W, fill, lane);
    if (groups && lane == 0 && g_culled) atomicAdd(&a.counters[C_GROUP], (unsigned long long)g_culled);
}

// ---------------------------------------------------------------------------
// k_cull_b: phase B over the survivor queue, warp-cooperative.  Each warp
// takes 32 survivors at a time: (1) per lane, range cull and azimuth span;
// large spans go to the deferred queue, small live spans whose candidate rays
// already hold closer hits are dropped (pair_occluded), the others go to the
// warp's list of pending pairs; (2) once 32 pairs are pending, one per lane
// gets its test setup into shared memory; (3) the warp expands and tests all
// candidates of those 32 pairs together, one candidate per lane (owner found
// from the warp's prefix sums), so the setups and tests run with full warps
// and without lane divergence.
// ---------------------------------------------------------------------------
struct CullBWarpSmem {
    float st[SETUP_FIELDS][32];  // field-major setups of the warp's 32 pairs
    uint32_t meta[32];           // per pair: first channel | ray count << 10 | sensor << 26
    uint32_t r0[32];             // per pair: first ray index (wrapped)
    uint32_t tri[32];            // per pair: triangle id
    float inv[32];               // per pair: rounded-up 1 / ray count
    uint32_t own[32];            // lane of the pair with the r-th candidate run (r-th set bit of the owner mask)
    uint4 pend[64];              // live pairs waiting for their setup: triangle, meta, first ray, candidates
    uint32_t cnt[9];             // live, cand, inl, big, tests, hits, unc, ties, occluded
};

// Tie check of a committed certain hit against the key its atomicMin
// returned (FP32 + re-test mode): a different triangle within the tie band
// queues both for the FP64 re-test.
__device__ __forceinline__ void tie_check(const CastArgs& a, uint32_t g, uint32_t tri, float t, unsigned long long old,
                                          uint32_t& n_ties) {
    const uint32_t oid = (uint32_t)old;
    if (oid != NO_HIT && oid != tri) {
        const float told = __uint_as_float((uint32_t)(old >> 32));
        if (fabsf(__fsub_rn(t, told)) <= __fmul_rn(BETA, fmaxf(t, told))) {
            push_recheck(a, g, tri, __fmul_rn(t, 1.f - TAU_T), UC_TIE);
            push_recheck(a, g, oid, __fmul_rn(told, 1.f - TAU_T), UC_TIE);
            n_ties++;
        }
    }
}

// Setup and cooperative candidate expansion of the warp's pending live pairs
// W.pend[0, np), np <= 32: one pair per lane gets its test setup into shared
// memory, then the warp tests all candidates of the np pairs together, one
// candidate per lane per round (owner found from the warp's prefix sums).
// (Testing each pair's first candidate by its setup lane measured 1 % slower
// on c5: a second inlined copy of the test and commit.)  The tie check of a
// commit waits for the next round, so that the atomicMin's returned key
// arrives while that round is tested.  Called by the whole warp.
template <bool RECHECK>
__device__ __forceinline__ void cull_b_test_pairs(const CastArgs& a, const CullSmem& M, CullBWarpSmem& W, uint32_t np,
                                                  uint32_t lane, bool dump, uint32_t& c_hits, uint32_t& c_unc,
                                                  uint32_t& c_ties) {
    uint32_t ncand = 0;
    // a committed hit waiting for its tie check
    bool pend = false;
    uint32_t pg = 0, ptri = 0;
    float pt = 0.f;
    unsigned long long pold = 0ull;
    if (lane < np) {
        const uint4 e = W.pend[lane];
        const uint32_t tri = e.x, meta = e.y, my_r0 = e.z, nc = e.w;
        const uint32_t sn = meta >> 26;
        const SensorDev& S = M.sens[sn];
        float t9[9];
        const float* src = a.tris + 9ull * tri;
#pragma unroll
        for (int k = 0; k < 9; ++k) t9[k] = __ldg(src + k);
        TriW T;
        tri_world(t9, T);
        V3 w[3], p[3];
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) {
            w[kk] = rel_origin(S, T.v[kk]);
            p[kk] = rotB(S.B, w[kk]);
        }
        const float det = vdot(w[0], T.n);
        const float err_det = det_error(w[0], T);
        const bool det_unc = fabsf(det) <= err_det;
        if (det != 0.f || (RECHECK && det_unc)) {
            make_setup(S, T, w, p, det, err_det, SetupWriterSoA{&W.st[0][0], lane});
            W.tri[lane] = tri;
            W.meta[lane] = meta;
            W.r0[lane] = my_r0;
            W.inv[lane] = __frcp_ru((float)((meta >> 10) & 0xFFFFu));
            ncand = nc;
        }
    }
    // warp prefix sum of the candidate counts
    uint32_t incl = ncand;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += t;
    }
    const uint32_t excl = incl - ncand;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t nz = __ballot_sync(0xffffffffu, ncand > 0);   // lanes that own candidates, in order
    if (ncand > 0) W.own[__popc(nz & ((1u << lane) - 1u))] = lane;
    if (lane == 0) {
        W.cnt[2] += total;
        W.cnt[4] += total;
    }
    __syncwarp();
    for (uint32_t c0 = 0; c0 < total; c0 += 32) {
        // rank (among owning lanes) of the pair holding candidate c0, and the
        // pairs that start inside this round of 32 candidates
        const uint32_t base_rank = __popc(__ballot_sync(0xffffffffu, ncand > 0 && incl <= c0));
        const uint32_t starts =
            __reduce_or_sync(0xffffffffu, (ncand > 0 && excl > c0 && excl < c0 + 32) ? (1u << (excl - c0)) : 0u);
        const uint32_t rank = base_rank + __popc(starts & ((2u << lane) - 2u));
        const uint32_t own = W.own[min(rank, 31u)];
        const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, own & 31u);
        const uint32_t meta = W.meta[own & 31u];
        const uint32_t r0o = W.r0[own & 31u];
        const uint32_t tri = W.tri[own & 31u];
        const float inv = W.inv[own & 31u];
        const uint32_t cc = c0 + lane;
        int res = T_MISS;
        float t = 0.f, terr = 0.f;
        uint32_t g = 0;
        unsigned long long cur = 0ull;
        if (cc < total) {
            const uint32_t nr = (meta >> 10) & 0xFFFFu;
            const uint32_t sn = meta >> 26;
            const uint32_t idx = cc - o_excl;
            // quotient from the rounded-up reciprocal, then one correction
            // step in each direction (enough for idx < 2^24, where (float)idx
            // is exact); a quotient still off (larger spans of the no-cull
            // debug mode, up to 1024 x 32768 candidates) takes the exact division
            uint32_t jo = (uint32_t)((float)idx * inv);
            if (jo * nr > idx) --jo;
            uint32_t io = idx - jo * nr;
            if (io >= nr) {
                ++jo;
                io -= nr;
            }
            if (io >= nr) {
                jo = idx / nr;
                io = idx - jo * nr;
            }
            const SensorDev& S = M.sens[sn];
            const uint32_t j = (meta & 1023u) + jo;
            uint32_t i = r0o + io;
            if (i >= S.n_rays) i -= S.n_rays;
            g = S.ray_off + j * S.n_rays + i;
            cur = __ldcg(&a.keys[g]);   // issued before the test arithmetic
            V3 d = ray_dir(M.ch[S.ch_loc + j], __ldg(&a.az_sc[S.az_off + i]));
            res = test_fp32<RECHECK>(SetupSoA{&W.st[0][0], own & 31u}, S, d, t, terr);
            if (dump) dump_candidate(a, g, tri);
        }
        if (RECHECK && pend) tie_check(a, pg, ptri, pt, pold, c_ties);
        pend = false;
        if (res == T_MISS) continue;
        const float tcur = __uint_as_float((uint32_t)(cur >> 32));
        if (is_uncertain(res)) {
            // a re-test can only change the result if it may beat the current best
            c_unc += queue_uncertain(a, g, tri, res, t, terr, W.st[21][own & 31u], tcur);
            continue;
        }
        c_hits++;
        const unsigned long long key = ((unsigned long long)__float_as_uint(t) << 32) | tri;
        if (!RECHECK) {
            if (key < cur) atomicMin(&a.keys[g], key);
        } else if (!(t > __fmul_rn(tcur, 1.f + BETA))) {
            pold = atomicMin(&a.keys[g], key);
            pend = true;
            pg = g;
            ptri = tri;
            pt = t;
        }
    }
    if (RECHECK && pend) tie_check(a, pg, ptri, pt, pold, c_ties);
    __syncwarp();
}

// A live pair with at most OCC_MAX candidate rays is dropped before its
// setup when every candidate ray already holds a certain hit (the keys hold
// only those) whose FP32 distance, widened by the tie band, lies below the
// pair's distance lower bound less the FP32 error of a certain t.  None of
// its candidates could then win, tie or be kept for the re-test: a certain
// hit of the pair would be farther than tcur (1 + BETA) and is never
// committed, and an uncertain one has a lower bound of at least t_lb, which
// queue_uncertain does not queue.  Keys only decrease, so the test loop
// would drop every candidate of the pair as well, and the result is the same
// bits.  The candidate keys are read (high words, L2) before they are compared.
// Casts that dump their candidates (a debug mode that checks the culls'
// superset) or pass GRCA_CAST_NO_OCCLUSION drop no pair this way.
constexpr uint32_t OCC_MAX = 4;
__device__ __forceinline__ bool pair_occluded(const CastArgs& a, const SensorDev& S, const V3 p[3], uint32_t j0,
                                              uint32_t r0, uint32_t n_r, uint32_t nc) {
    const float lb = pair_t_lb(p);
    if (!(lb > 0.f)) return false;
    const float thr = __fmul_rn(lb, 1.f - 2.f * TAU_T);
    const unsigned int* hw = reinterpret_cast<const unsigned int*>(a.keys) + 1;   // t bits of key g at 2g + 1
    float tk[OCC_MAX];
    uint32_t j = j0, i = r0, io = 0;
#pragma unroll
    for (uint32_t q = 0; q < OCC_MAX; ++q) {
        tk[q] = 0.f;
        if (q < nc) {
            tk[q] = __uint_as_float(__ldcg(hw + 2ull * (S.ray_off + j * S.n_rays + i)));
            if (++i == S.n_rays) i = 0;
            if (++io == n_r) {
                io = 0;
                ++j;
                i = r0;
            }
        }
    }
    bool occ = true;
#pragma unroll
    for (uint32_t q = 0; q < OCC_MAX; ++q)
        if (q < nc) occ = occ && thr > __fmul_rn(tk[q], 1.f + BETA);
    return occ;
}

template <bool RECHECK, bool BRUTE>
__global__ void __launch_bounds__(256, 4) k_cull_b(CastArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    CullSmem M = cull_smem_prologue(a, smem, false);
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    CullBWarpSmem& W = reinterpret_cast<CullBWarpSmem*>(M.rest)[wib];
    const bool dump = a.flags & 16u;
    if (lane < 9) W.cnt[lane] = 0;
    __syncwarp();
    uint32_t c_unc = 0, c_ties = 0, c_hits = 0;
    const uint32_t n = min(*(volatile uint32_t*)&a.qcount[Q_SURV], a.surv_cap);
    // part 1 records how far it goes; part 2 starts there (a.surv_part)
    const uint32_t s0 = a.surv_part == 2 ? min(*(volatile uint32_t*)&a.qcount[Q_SURV_SPLIT], n) : 0u;
    if (a.surv_part == 1 && blockIdx.x == 0 && threadIdx.x == 0) a.qcount[Q_SURV_SPLIT] = n;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t gwarp = ((blockIdx.x * blockDim.x) >> 5) + wib;
    // Live pairs with small spans queue up in W.pend and get their setups 32
    // at a time, so that the setup and the tests run with full warps even
    // where the azimuth cull or the deferred queue took many of a batch's
    // survivors (warp-uniform count)
    uint32_t fill = 0;
    for (uint32_t b0 = s0 + gwarp * 32; b0 < n; b0 += n_warps * 32) {
        const uint32_t q = b0 + lane;
        uint32_t l_live = 0, l_cand = 0, l_big = 0, l_occ = 0;
        bool pend_me = false;
        uint4 pe = make_uint4(0u, 0u, 0u, 0u);
        if (q < n) {
            const unsigned long long r = __ldcs(&a.surv[q]);
            const uint32_t tri = (uint32_t)r, span = (uint32_t)(r >> 32) & 0x1FFFFFu, sn = (uint32_t)(r >> 53);
            const SensorDev& S = M.sens[sn];
            float t9[9];
            const float* src = a.tris + 9ull * tri;
#pragma unroll
            for (int k = 0; k < 9; ++k) t9[k] = __ldg(src + k);
            V3 vv[3] = {{t9[0], t9[1], t9[2]}, {t9[3], t9[4], t9[5]}, {t9[6], t9[7], t9[8]}};
            V3 w[3], p[3];
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                w[kk] = rel_origin(S, vv[kk]);
                p[kk] = rotB(S.B, w[kk]);
            }
            bool keep = true;
            if (!BRUTE && S.has_range) {
                // range cull (App. A.4.1 Step 1), only where provably empty
                float dmax2 = fmaxf(vdot(w[0], w[0]), fmaxf(vdot(w[1], w[1]), vdot(w[2], w[2])));
                float dlo = fmaxf(S.d_min * (1.f - 1e-5f) - 1e-6f, 0.f);
                if (dmax2 < dlo * dlo) keep = false;
                const float dhi = S.d_max * (1.f + 1e-5f) + 1e-6f;
                // the closest point matters only if some vertex lies beyond d_max
                if (keep && S.d_max < INFINITY && dmax2 > dhi * dhi && closest_dist(w[0], w[1], w[2]) > dhi)
                    keep = false;
            }
            Span sp;
            sp.j_lo = (int)(span & 1023u);
            sp.j_hi = (int)((span >> 10) & 1023u);
            sp.pierced = (span >> 20) & 1u;
            if (keep) {
                if (BRUTE) {
                    sp.u_lo = 0;
                    sp.n_r = (int)S.n_rays;
                    sp.a0 = 0.f;
                } else {
                    sp.a0 = ray_units(S, fast_atan2(p[0].y, p[0].x));
                    float A, B;
                    if (sp.pierced) {
                        A = sp.a0 - 0.5f * S.period;
                        B = sp.a0 + 0.5f * S.period;
                    } else {
                        float d1 = rel_angle(p[0], p[1]);
                        float d2 = rel_angle(p[0], p[2]);
                        float pad = EPS_T + 3.f * FAST_ATAN_PAD + az_pad2(p[0]) + az_pad2(p[1]) + az_pad2(p[2]);
                        float lo = fminf(0.f, fminf(d1, d2)) - pad, hi = fmaxf(0.f, fmaxf(d1, d2)) + pad;
                        if (hi - lo >= 6.2831f) {
                            A = sp.a0 - 0.5f * S.period;
                            B = sp.a0 + 0.5f * S.period;
                        } else {
                            A = sp.a0 + lo * S.inv_dtheta;
                            B = sp.a0 + hi * S.inv_dtheta;
                        }
                    }
                    keep = ray_interval(S, A - PADR - S.az_noise_pad, B + PADR + S.az_noise_pad, sp.u_lo, sp.n_r);
                }
            }
            if (keep) {
                const uint32_t nc = (uint32_t)(sp.j_hi - sp.j_lo + 1) * (uint32_t)sp.n_r;
                l_live = 1;
                l_cand = nc;
                if (!BRUTE && nc > a.inline_max) {
                    cg::coalesced_group grp = cg::coalesced_threads();
                    uint32_t bb = 0;
                    if (grp.thread_rank() == 0) bb = atomicAdd(&a.qcount[Q_BIG], grp.size());
                    bb = grp.shfl(bb, 0) + grp.thread_rank();
                    if (bb < a.big_cap) {
                        BigPair bp;
                        bp.tri = tri;
                        bp.sensor = (uint16_t)sn;
                        bp.flags = sp.pierced ? 1 : 0;
                        bp.j_lo = (uint16_t)sp.j_lo;
                        bp.j_hi = (uint16_t)sp.j_hi;
                        bp.u_lo = sp.u_lo;
                        bp.n_r = (uint32_t)sp.n_r;
                        bp.a0 = sp.a0;
                        bp.pad_[0] = bp.pad_[1] = 0;
                        a.big[bb] = bp;
                    } else {
                        atomicOr(a.error, (uint32_t)ERR_BIG_CAP);
                    }
                    l_big = 1;
                } else {
                    const uint32_t r0 = (uint32_t)imod(sp.u_lo, (int)S.n_rays);
                    if (RECHECK && !BRUTE && !dump && !(a.flags & (uint32_t)GRCA_CAST_NO_OCCLUSION) &&
                        nc <= OCC_MAX &&
                        pair_occluded(a, S, p, (uint32_t)sp.j_lo, r0, (uint32_t)sp.n_r, nc)) {
                        l_occ = 1;
                    } else {
                        pend_me = true;
                        pe = make_uint4(tri, (uint32_t)sp.j_lo | ((uint32_t)sp.n_r << 10) | (sn << 26), r0, nc);
                    }
                }
            }
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, pend_me);
        if (pend_me) W.pend[fill + __popc(bal & ((1u << lane) - 1u))] = pe;   // fill < 32 here: index < 64
        fill += __popc(bal);
        {
            const uint32_t s_live = __reduce_add_sync(0xffffffffu, l_live), s_cand = __reduce_add_sync(0xffffffffu, l_cand),
                           s_big = __reduce_add_sync(0xffffffffu, l_big), s_occ = __reduce_add_sync(0xffffffffu, l_occ);
            if (lane == 0) {
                W.cnt[0] += s_live;
                W.cnt[1] += s_cand;
                W.cnt[3] += s_big;
                W.cnt[8] += s_occ;
            }
        }
        __syncwarp();
        if (fill >= 32u) {
            cull_b_test_pairs<RECHECK>(a, M, W, 32u, lane, dump, c_hits, c_unc, c_ties);
            if (lane + 32u < fill) W.pend[lane] = W.pend[lane + 32u];
            __syncwarp();
            fill -= 32u;
        }
    }
    if (fill > 0u) cull_b_test_pairs<RECHECK>(a, M, W, fill, lane, dump, c_hits, c_unc, c_ties);
    c_unc = __reduce_add_sync(0xffffffffu, c_unc);
    c_ties = __reduce_add_sync(0xffffffffu, c_ties);
    c_hits = __reduce_add_sync(0xffffffffu, c_hits);
    __syncwarp();
    if (lane == 0) {
        const int idx[9] = {C_PAIRS_LIVE, C_CAND, C_CAND_INLINE, C_BIG, C_TESTS, C_HITS, C_UNCERTAIN, C_TIES, C_OCCLUDED};
        W.cnt[5] += c_hits;
        W.cnt[6] = c_unc;
        W.cnt[7] = c_ties;
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (W.cnt[k]) atomicAdd(&a.counters[idx[k]], (unsigned long long)W.cnt[k]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.counters[C_SURV] = *(volatile uint32_t*)&a.qcount[Q_SURV];
}

// ---------------------------------------------------------------------------
// per-channel azimuth span of a deferred pair (cone/plane crossings)
// ---------------------------------------------------------------------------
// Relative azimuth (to vertex 0) of every crossing of channel level s (sin)
// with the triangle's edges: the quadratic of Sec. 3.5.2
// (a_z + l e_z)^2 c^2 - s^2 |a_h + l e_h|^2 = 0 on the forward nappe, or the
// plane case of Sec. 3.5.1 for s == 0.  Returns false if no edge crosses.
__device__ __forceinline__ bool channel_span_rel(const V3 p[3], const float s_v[3], float s, float c, float& lo,
                                                 float& hi) {
    bool any = false;
    lo = 1e30f;
    hi = -1e30f;
    V3 p0 = p[0];
    auto include = [&](V3 q, float extra) {
        float ang = rel_angle(p0, q);
        float pad = EPS_ROW + FAST_ATAN_PAD + az_pad(q) + extra;
        lo = fminf(lo, ang - pad);
        hi = fmaxf(hi, ang + pad);
        any = true;
    };
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        V3 a = p[k], b = p[k == 2 ? 0 : k + 1];
        float emin = fminf(s_v[k], s_v[k == 2 ? 0 : k + 1]), emax = fmaxf(s_v[k], s_v[k == 2 ? 0 : k + 1]);
        edge_elev_extremum(a, b, emin, emax);
        if (s < emin - EPS_S || s > emax + EPS_S) continue;
        V3 e = {b.x - a.x, b.y - a.y, b.z - a.z};
        bool found = false;
        if (s == 0.f) {
            if (a.z == 0.f && b.z == 0.f) {
                include(a, 0.f);
                include(b, 0.f);
                found = true;
            } else if ((a.z <= 0.f && b.z >= 0.f) || (a.z >= 0.f && b.z <= 0.f)) {
                float lam = a.z / (a.z - b.z);
                V3 q = {a.x + lam * e.x, a.y + lam * e.y, a.z + lam * e.z};
                include(q, 0.f);
                found = true;
            }
        } else {
            float c2 = c * c, s2 = s * s;
            float A = e.z * e.z * c2 - s2 * (e.x * e.x + e.y * e.y);
            float Bh = a.z * e.z * c2 - s2 * (a.x * e.x + a.y * e.y);
            float C = a.z * a.z * c2 - s2 * (a.x * a.x + a.y * a.y);
            float lam[2];
            int nl = 0;
            float scaleA = e.z * e.z * c2 + s2 * (e.x * e.x + e.y * e.y);
            if (fabsf(A) <= 1e-5f * scaleA) {
                if (Bh != 0.f) lam[nl++] = -C / (2.f * Bh);
            } else {
                float disc = Bh * Bh - A * C;
                if (disc >= 0.f) {
                    float sq = sqrtf(disc);
                    float qq = -(Bh + copysignf(sq, Bh));
                    lam[nl++] = qq / A;
                    if (qq != 0.f) lam[nl++] = C / qq;
                } else if (disc > -1e-3f * Bh * Bh) {
                    lam[nl++] = -Bh / A;  // tangent touch
                }
            }
            for (int r = 0; r < nl; ++r) {
                float l = lam[r];
                if (!(l >= -1e-4f && l <= 1.0001f)) continue;
                l = fminf(fmaxf(l, 0.f), 1.f);
                V3 q = {a.x + l * e.x, a.y + l * e.y, a.z + l * e.z};
                float qr = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z);
                if ((s > 0.f && q.z < -1e-5f * qr) || (s < 0.f && q.z > 1e-5f * qr)) continue;  // mirror nappe
                include(q, 0.f);
                found = true;
            }
        }
        if (!found) {  // numerics gave no usable root although the edge spans the level
            include(a, 0.f);
            include(b, 0.f);
        }
    }
    return any;
}

__global__ void __launch_bounds__(256) k_expand(CastArgs a) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t n_big = min(*(volatile uint32_t*)&a.qcount[Q_BIG], a.big_cap);
    const uint32_t CH = a.chunk_rays;
    for (uint32_t bp = gw; bp < n_big; bp += nw) {
        BigPair P = a.big[bp];
        const SensorDev& S = a.sensors[P.sensor];
        TriW T;
        float t9[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) t9[q] = __ldg(&a.tris[9ull * P.tri + q]);
        tri_world(t9, T);
        V3 w[3], p[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            w[k] = rel_origin(S, T.v[k]);
            p[k] = rotB(S.B, w[k]);
        }
        float det = vdot(w[0], T.n);
        float err_det = det_error(w[0], T);
        if (lane == 0) {
            PairSetup st;
            make_setup(S, T, w, p, det, err_det, SetupWriterAoS{st});
            a.setups[bp] = st;
        }
        float s_v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float r2 = p[k].x * p[k].x + p[k].y * p[k].y + p[k].z * p[k].z;
            s_v[k] = r2 > 0.f ? p[k].z * rsqrtf(r2) : 0.f;
        }
        const int n = (int)S.n_rays;
        const bool full_pair = P.n_r >= (uint32_t)n;
        for (int jb = P.j_lo; jb <= (int)P.j_hi; jb += 32) {
            int j = jb + (int)lane;
            uint32_t nch = 0;
            int r_first = 0, cnt = 0;
            if (j <= (int)P.j_hi) {
                int u_lo = P.u_lo, n_r = (int)P.n_r;
                if (!(P.flags & 1u)) {
                    float2 sc = a.ch_sc[S.ch_off + j];
                    float lo, hi;
                    if (channel_span_rel(p, s_v, sc.x, sc.y, lo, hi)) {
                        int ru, rn;
                        if (hi - lo < 6.2831f &&
                            ray_interval(S, P.a0 + lo * S.inv_dtheta - PADR - S.az_noise_pad,
                                         P.a0 + hi * S.inv_dtheta + PADR + S.az_noise_pad, ru, rn)) {
                            if (full_pair) {
                                u_lo = ru;
                                n_r = rn;
                            } else {
                                int l2 = max(ru, u_lo), h2 = min(ru + rn - 1, u_lo + n_r - 1);
                                u_lo = l2;
                                n_r = h2 - l2 + 1;
                            }
                        } else if (!(hi - lo < 6.2831f)) {
                            // keep the pair span
                        } else {
                            n_r = 0;
                        }
                    } else {
                        n_r = 0;
                    }
                }
                if (n_r > 0) {
                    cnt = n_r;
                    r_first = imod(u_lo, n);
                    nch = (uint32_t)((cnt + (int)CH - 1) / (int)CH);
                }
            }
            // warp prefix sum of chunk counts -> one atomic per warp
            uint32_t incl = nch;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += v;
            }
            uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            if (total == 0) continue;
            uint32_t b0 = 0;
            if (lane == 0) b0 = atomicAdd(&a.qcount[Q_CHUNK], total);
            b0 = __shfl_sync(0xffffffffu, b0, 0) + incl - nch;
            for (uint32_t q = 0; q < nch; ++q) {
                uint32_t idx = b0 + q;
                if (idx < a.chunk_cap) {
                    int r = r_first + (int)(q * CH);
                    if (r >= n) r -= n;
                    a.chunks[idx] = make_uint4(bp, (uint32_t)j, (uint32_t)r, (uint32_t)min((int)CH, cnt - (int)(q * CH)));
                } else {
                    atomicOr(a.error, (uint32_t)ERR_CHUNK_CAP);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// k_test: one warp per chunk of one (pair, channel) row
// ---------------------------------------------------------------------------
template <bool RECHECK>
__global__ void __launch_bounds__(256, 4) k_test(CastArgs a) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    const uint32_t n_chunks = min(*(volatile uint32_t*)&a.qcount[Q_CHUNK], a.chunk_cap);
    const bool dump = a.flags & 16u;
    const bool occl = RECHECK && !dump && !(a.flags & (uint32_t)GRCA_CAST_NO_OCCLUSION);
    uint32_t c_tests = 0, c_hits = 0, c_unc = 0, c_ties = 0;
    for (uint32_t c = gw; c < n_chunks; c += nw) {
        uint4 ck = a.chunks[c];
        const uint32_t bp = ck.x, j = ck.y, r0 = ck.z, cnt = ck.w;
        const uint32_t tri = a.big[bp].tri;
        const SensorDev& S = a.sensors[a.big[bp].sensor];
        const PairSetup st = a.setups[bp];
        const uint32_t n = S.n_rays;
        const float2 chv = a.ch_sc[S.ch_off + j];
        const uint32_t gbase = S.ray_off + j * n;
        for (uint32_t q = lane; q < cnt; q += 32) {
            uint32_t i = r0 + q;
            if (i >= n) i -= n;
            // a candidate whose ray already holds a certain hit closer than the
            // pair's distance lower bound by more than the tie band is dropped,
            // as in k_cull_b (the same bits)
            const unsigned long long cur = __ldcg(&a.keys[gbase + i]);
            if (occl && __fmul_rn(st.t_lb, 1.f - 2.f * TAU_T) >
                            __fmul_rn(__uint_as_float((uint32_t)(cur >> 32)), 1.f + BETA))
                continue;
            V3 d = ray_dir(chv, __ldg(&a.az_sc[S.az_off + i]));
            float t, terr;
            int res = test_fp32<RECHECK>(SetupAoS{st}, S, d, t, terr);
            c_tests++;
            if (dump) dump_candidate(a, gbase + i, tri);
            c_hits += commit_pre<RECHECK>(a, gbase + i, tri, res, t, terr, st.t_lb, cur, c_unc, c_ties);
        }
    }
    warp_add(&a.counters[C_TESTS], c_tests);
    warp_add(&a.counters[C_HITS], c_hits);
    warp_add(&a.counters[C_UNCERTAIN], c_unc);
    warp_add(&a.counters[C_TIES], c_ties);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.counters[C_CHUNKS] = *(volatile uint32_t*)&a.qcount[Q_CHUNK];
    }
}

// ---------------------------------------------------------------------------
// FP64 re-test (world frame, same watertight edge-function formulation)
// ---------------------------------------------------------------------------
struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 dsub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double ddot(D3 a, D3 b) { return __fma_rn(a.x, b.x, __fma_rn(a.y, b.y, __dmul_rn(a.z, b.z))); }
__device__ __forceinline__ D3 dcross(D3 a, D3 b) {
    return {__dsub_rn(__dmul_rn(a.y, b.z), __dmul_rn(a.z, b.y)), __dsub_rn(__dmul_rn(a.z, b.x), __dmul_rn(a.x, b.z)),
            __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x))};
}

__device__ __forceinline__ void decode_ray(const CastArgs& a, uint32_t g, uint32_t& sn, uint32_t& j, uint32_t& i) {
    sn = 0;
    for (uint32_t k = 1; k < a.n_sensors; ++k)
        if (a.sensors[k].ray_off <= g) sn = k;
    const SensorDev& S = a.sensors[sn];
    uint32_t loc = g - S.ray_off;
    j = loc / S.n_rays;
    i = loc - j * S.n_rays;
}

// returns the u64 key of the FP64 result (KEY_MISS on a miss).  edges =
// false skips the edge functions: for a (ray, triangle) pair that the FP32
// test found inside every edge with margin (a certain hit, or an entry
// uncertain only in t or in the range), whose FP64 edge functions are
// positive too; every other step is the same, so the key is the same bits.
__device__ unsigned long long test_fp64(const CastArgs& a, uint32_t g, uint32_t tri, bool edges = true) {
    uint32_t sn, j, i;
    decode_ray(a, g, sn, j, i);
    const SensorDev& S = a.sensors[sn];
    double2 ch = a.ch_sc64[S.ch_off + j];
    double2 az = a.az_sc64[S.az_off + i];
    double ca = az.y * ch.y, sa = az.x * ch.y, su = ch.x;
    D3 d = {ca * S.B64[0] + sa * S.B64[3] + su * S.B64[6], ca * S.B64[1] + sa * S.B64[4] + su * S.B64[7],
            ca * S.B64[2] + sa * S.B64[5] + su * S.B64[8]};
    const float* t9 = a.tris + 9ull * tri;
    const V3 f0 = {__ldg(t9 + 0), __ldg(t9 + 1), __ldg(t9 + 2)}, f1 = {__ldg(t9 + 3), __ldg(t9 + 4), __ldg(t9 + 5)},
             f2 = {__ldg(t9 + 6), __ldg(t9 + 7), __ldg(t9 + 8)};
    const D3 v0 = {(double)f0.x, (double)f0.y, (double)f0.z}, v1 = {(double)f1.x, (double)f1.y, (double)f1.z},
             v2 = {(double)f2.x, (double)f2.y, (double)f2.z};
    const D3 o = {S.o64[0], S.o64[1], S.o64[2]};
    const D3 w0 = dsub(v0, o), w1 = dsub(v1, o), w2 = dsub(v2, o);
    D3 n = dcross(dsub(v1, v0), dsub(v2, v0));
    if (n.x == 0.0 && n.y == 0.0 && n.z == 0.0) return KEY_MISS;
    double det = ddot(w0, n);
    if (det == 0.0) return KEY_MISS;
    if ((a.flags & 2u) && det > 0.0) return KEY_MISS;  // back-facing
    double fold = det < 0.0 ? -1.0 : 1.0;
    // canonical edge functions (same rule as the FP32 test): base = the
    // lexicographically smaller vertex, evaluated from it; selects, no arrays
#pragma unroll
    for (int k = 0; k < 3 && edges; ++k) {
        const V3 fa = k == 0 ? f0 : (k == 1 ? f1 : f2), fb = k == 0 ? f1 : (k == 1 ? f2 : f0);
        const D3 va = k == 0 ? v0 : (k == 1 ? v1 : v2), vb = k == 0 ? v1 : (k == 1 ? v2 : v0);
        const D3 wa = k == 0 ? w0 : (k == 1 ? w1 : w2), wb = k == 0 ? w1 : (k == 1 ? w2 : w0);
        const bool fwd = !lex_less(fb, fa);
        const D3 wbase = fwd ? wa : wb, vbase = fwd ? va : vb, voth = fwd ? vb : va;
        const D3 m = dcross(wbase, dsub(voth, vbase));
        double E = ddot(d, m) * (fwd ? fold : -fold);
        if (E < 0.0) return KEY_MISS;
    }
    double dn = ddot(d, n);
    if (dn == 0.0) return KEY_MISS;
    double t = det / dn;
    if (!(t > 0.0) || t < S.d_min64 || t > S.d_max64) return KEY_MISS;
    float tf = __double2float_rn(t);
    return ((unsigned long long)__float_as_uint(tf) << 32) | tri;
}

// R-1: the queued entries uncertain only in t (cause UC_T) get t re-evaluated
// in double-float (refine_t).  A settled hit is committed like a certain FP32
// hit (key minimum, tie detection against the returned key) and its entry
// retired (triangle NO_HIT); a settled miss is retired; an entry still
// uncertain stays for the FP64 re-test.  Runs after every FP32 test of the
// frame, before the filter, so the commit order does not matter: the tie
// chain of the FP32 commits holds for any order.
// the queue length k_refine works on, taken by the launch before it: k_refine
// appends tie entries to the same queue, and a block that started late would
// otherwise count slots reserved by other blocks but not written yet
__global__ void k_refine_count(CastArgs a) { a.qcount[Q_REFINE_N] = *(volatile uint32_t*)&a.qcount[Q_RECHECK]; }

__global__ void k_refine(CastArgs a) {
    const uint32_t np = min(a.qcount[Q_REFINE_N], a.recheck_cap);
    uint32_t n_ref = 0, n_hit = 0, n_ties = 0;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < np; q += gridDim.x * blockDim.x) {
        const uint4 e = a.recheck[q];
        if (e.w != (uint32_t)UC_T) continue;
        uint32_t sn, j, i;
        decode_ray(a, e.x, sn, j, i);
        const Refined rf = refine_t(a, a.sensors[sn], j, i, e.y);
        n_ref++;
        if (rf.res == T_UNCERTAIN + UC_T) continue;
        if (rf.res == T_UNCERTAIN + UC_RANGE) {
            a.recheck[q] = make_uint4(e.x, e.y, __float_as_uint(__fmul_rn(rf.t, __fsub_rn(1.f, rf.e))), UC_RANGE);
            continue;
        }
        a.recheck[q].y = NO_HIT;  // retired: settled here
        if (rf.res != T_HIT) continue;
        n_hit++;
        const float t = rf.t;
        unsigned long long* kp = &a.keys[e.x];
        const float tcur = __uint_as_float((uint32_t)(__ldcg(kp) >> 32));
        if (t > __fmul_rn(tcur, 1.f + BETA)) continue;
        const unsigned long long key = ((unsigned long long)__float_as_uint(t) << 32) | e.y;
        const unsigned long long old = atomicMin(kp, key);
        const uint32_t oid = (uint32_t)old;
        if (oid != NO_HIT && oid != e.y) {
            const float told = __uint_as_float((uint32_t)(old >> 32));
            if (fabsf(__fsub_rn(t, told)) <= __fmul_rn(BETA, fmaxf(t, told))) {
                push_recheck(a, e.x, e.y, __fmul_rn(t, 1.f - TAU_T), UC_TIE);
                push_recheck(a, e.x, oid, __fmul_rn(told, 1.f - TAU_T), UC_TIE);
                n_ties++;
            }
        }
    }
    warp_add(&a.counters[C_REFINED], n_ref);
    warp_add(&a.counters[C_HITS], n_hit);
    warp_add(&a.counters[C_TIES], n_ties);
}

// R0: keep the queued pairs that can still beat or tie the ray's final FP32
// winner (t_lo <= t_best (1 + beta)); flag their rays; drop the rest.  A kept
// pair whose triangle is the ray's FP32 winner is flagged but not kept: R1
// re-tests the winner of every flagged ray, so R2 would repeat that test.
// Also counts the queued and the kept entries per cause (UC_*).
__global__ void k_recheck_filter(CastArgs a) {
    uint32_t np = min(*(volatile uint32_t*)&a.qcount[Q_RECHECK], a.recheck_cap);
    uint32_t nq[UC_NUM] = {}, nk[UC_NUM] = {};
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < np; q += gridDim.x * blockDim.x) {
        uint4 e = a.recheck[q];
        const unsigned long long kb = a.keys[e.x];
        // a sharded cast compares against the winner over every shard
        float tbest = __uint_as_float((uint32_t)((a.keys_glob ? a.keys_glob[e.x] : kb) >> 32));
        // entries retired by k_refine count as queued, never as kept
        const bool kept = e.y != NO_HIT && __uint_as_float(e.z) <= __fmul_rn(tbest, 1.f + BETA);
#pragma unroll
        for (int k = 0; k < UC_NUM; ++k) {
            nq[k] += e.w == (uint32_t)k;
            nk[k] += kept && e.w == (uint32_t)k;
        }
        if (kept) {
            flag_ray(a, e.x);
            if (e.y == (uint32_t)kb) a.recheck[q].y = NO_HIT;
        } else if (e.y != NO_HIT) {
            a.recheck[q].y = NO_HIT;
        }
    }
#pragma unroll
    for (int k = 0; k < UC_NUM; ++k) {
        warp_add(&a.counters[C_QUEUED0 + k], nq[k]);
        warp_add(&a.counters[C_KEPT0 + k], nk[k]);
    }
}

// R1: every flagged ray starts from the FP64 result of its FP32 winner
__global__ void k_recheck_rays(CastArgs a) {
    uint32_t nf = min(*(volatile uint32_t*)&a.qcount[Q_FLAG], a.flag_cap);
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nf; q += gridDim.x * blockDim.x) {
        uint32_t g = a.flag_list[q];
        unsigned long long k = a.keys[g];
        uint32_t id = (uint32_t)k;
        // the FP32 winner is a certain hit: inside every edge with margin
        a.keys64[g] = id == NO_HIT ? KEY_MISS : test_fp64(a, g, id, false);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) a.counters[C_FLAGGED] = *(volatile uint32_t*)&a.qcount[Q_FLAG];
}

constexpr int RECHECK_BLOCK = 256;

// R2: FP64 re-test of every kept (ray, triangle) pair.  The FP64 pipe runs
// at a small fraction of the FP32 rate, and a warp pays for a test however
// few of its lanes take part, so each warp first compacts the kept pairs of
// its slices of the queue into shared memory and tests them 32 at a time.
// pr.x: ray | bit 31 set when the entry needs the FP64 edge functions (cause
// edge or orientation; ray ids stay below 2^31: 64 sensors x 1024 x 32768)
__device__ __forceinline__ void recheck_pair(const CastArgs& a, uint2 pr) {
    const uint32_t g = pr.x & 0x7FFFFFFFu;
    const unsigned long long k = test_fp64(a, g, pr.y, (pr.x >> 31) != 0u);
    if (k != KEY_MISS) atomicMin(&a.keys64[g], k);
}
__global__ void __launch_bounds__(RECHECK_BLOCK) k_recheck_pairs(CastArgs a) {
    __shared__ uint2 buf[RECHECK_BLOCK / 32][64];
    const uint32_t lane = threadIdx.x & 31u;
    uint2* wb = buf[threadIdx.x >> 5];
    const uint32_t np = min(*(volatile uint32_t*)&a.qcount[Q_RECHECK], a.recheck_cap);
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    uint32_t fill = 0, kept = 0;   // warp-uniform
    for (uint32_t q0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32u; q0 < np; q0 += n_warps * 32u) {
        const uint32_t q = q0 + lane;
        uint2 pr = make_uint2(0u, NO_HIT);
        if (q < np) {
            const uint4 e = a.recheck[q];
            const bool edges = e.w == (uint32_t)UC_EDGE || e.w == (uint32_t)UC_ORIENT;
            pr = make_uint2(e.x | (edges ? 0x80000000u : 0u), e.y);
        }
        const bool keep = pr.y != NO_HIT;
        const uint32_t bal = __ballot_sync(0xffffffffu, keep);
        if (keep) wb[fill + __popc(bal & ((1u << lane) - 1u))] = pr;   // fill < 32 here: index < 64
        fill += __popc(bal);
        __syncwarp();
        if (fill >= 32u) {
            recheck_pair(a, wb[lane]);
            __syncwarp();
            if (lane + 32u < fill) wb[lane] = wb[lane + 32u];
            __syncwarp();
            fill -= 32u;
            kept += 32u;
        }
    }
    if (lane < fill) recheck_pair(a, wb[lane]);
    kept += fill;
    if (lane == 0 && kept) atomicAdd(&a.counters[C_RECHECK], (unsigned long long)kept);
}

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// triangle-sharded casts (each GPU holds a slice of the triangles): the
// closest hit over the union of the slices is the key minimum over the
// slices' closest hits (Sec. 1.1, Eq. brute: a minimum over triangles),
// exchanged as one per-ray u64 MIN.  The FP64 re-test of a shard runs against
// the winner over all shards; a ray any shard flags is settled in FP64 by
// every shard that holds a candidate within its tie band, so that the last
// exchange (MIN of the settled keys) compares FP64 results wherever FP32
// cannot decide.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long rebase_key(unsigned long long k, uint32_t base) {
    const uint32_t id = (uint32_t)k;
    return id == NO_HIT ? k : ((k & 0xFFFFFFFF00000000ull) | (unsigned long long)(id + base));
}
__device__ __forceinline__ float key_t(unsigned long long k) { return __uint_as_float((uint32_t)(k >> 32)); }

// Stage 2a: the filter against the winner over all shards has flagged this
// shard's rays with kept queue entries; a ray whose own FP32 winner is not
// that winner but lies within its tie band is flagged as well.  Exported as
// one byte per ray for the MAX exchange.
__global__ void k_shard_flags(CastArgs a) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < a.n_rays_total; g += stride) {
        const unsigned long long kl = a.keys[g], kg = a.keys_glob[g];
        bool f = (a.flag_bits[g >> 5] >> (g & 31u)) & 1u;
        if (!f && (uint32_t)kl != NO_HIT && rebase_key(kl, a.tri_base) != kg &&
            key_t(kl) <= __fmul_rn(key_t(kg), 1.f + BETA))
            f = true;
        a.flags_out[g] = f ? 1 : 0;
    }
}

// Stage 2b: a ray some shard flagged is re-tested here too when this shard's
// FP32 winner lies within the tie band of the winner over all shards (the
// shard that holds that winner included), so that the final MIN compares FP64
// results only.
__global__ void k_shard_join(CastArgs a) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < a.n_rays_total; g += stride) {
        if (!a.flags_any[g]) continue;
        const unsigned long long kl = a.keys[g];
        if ((uint32_t)kl == NO_HIT || (a.flag_bits[g >> 5] >> (g & 31u)) & 1u) continue;
        if (key_t(kl) <= __fmul_rn(key_t(a.keys_glob[g]), 1.f + BETA)) flag_ray(a, g);
    }
}

// the shard's keys with global triangle ids (base + local id); resolved: the
// FP64 key for flagged rays
__global__ void k_shard_export(CastArgs a, uint32_t base, int resolved) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < a.n_rays_total; g += stride) {
        unsigned long long k = a.keys[g];
        if (resolved && (a.flag_bits[g >> 5] >> (g & 31u) & 1u)) k = a.keys64[g];
        a.keys_out[g] = rebase_key(k, base);
    }
}

// output function of SplitMix64 (Steele, Lea and Flood, 2014) for state x
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Post-processing of one ray (App. A.3 masks, App. A.1 range noise): a ray
// that does not fire reports a miss; a hit gets sigma * z added, z a
// Box-Muller normal from two counter-based uniforms of the ray's index.
__device__ __forceinline__ void post_ray(const CastArgs& a, uint32_t g, float& dist, uint32_t& id) {
    uint32_t sn = 0;
    for (uint32_t k = 1; k < a.n_sensors; ++k)
        if (a.sensors[k].ray_off <= g) sn = k;
    const SensorDev& S = a.sensors[sn];
    const uint32_t q = g - S.ray_off;
    if (S.mask && !((S.mask[q >> 5] >> (q & 31u)) & 1u)) {
        dist = __uint_as_float(0x7F800000u);
        id = NO_HIT;
        return;
    }
    if (S.range_sigma > 0.f && id != NO_HIT) {
        const unsigned long long c = S.noise_seed + 2ull * q;
        const float u1 = (float)((splitmix64(c) >> 40) + 1ull) * 5.9604645e-08f;  // (0, 1]
        const float u2 = (float)(splitmix64(c + 1ull) >> 40) * 5.9604645e-08f;    // [0, 1)
        dist += S.range_sigma * (sqrtf(-2.f * logf(u1)) * cospif(2.f * u2));
    }
}

// R3 fused into decode: flagged rays take the FP64 key
__global__ void k_decode(CastArgs a, int recheck) {
    uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < a.n_rays_total; g += stride) {
        unsigned long long k = a.keys[g];
        if (recheck && (a.flag_bits[g >> 5] >> (g & 31u) & 1u)) k = a.keys64[g];
        float dist = __uint_as_float((uint32_t)(k >> 32));
        uint32_t id = (uint32_t)k;
        if (a.post) post_ray(a, g, dist, id);
        a.out_dist[g] = dist;
        a.out_tri[g] = id;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        a.counters[C_PAIRS] = (unsigned long long)(a.n_tris - a.tri_first) * a.n_sensors;
}

// ---------------------------------------------------------------------------
// k_bvh: the static side of the hybrid static/dynamic pipeline (Sec. 7).
// A warp takes 32 consecutive rays (32 adjacent azimuths of one channel, a
// thin fan) and walks the static hierarchy once for all of them: every lane
// tests its own ray against both child boxes, and the warp enters a child
// if any lane's ray does (the nearer one first, by majority), keeping the
// other on a per-warp stack in shared memory.  At a leaf every lane tests
// its ray against the leaf's triangles: a cheap world-frame pre-test, then,
// for the few that pass, the culled path's own pair setup, FP32 test and
// closest-hit commit, into the same u64 keys, so static and dynamic results
// merge on the GPU by the key minimum.  Each lane skips subtrees that start
// beyond its best certain hit (dynamic or static, plus the tie band).
// ---------------------------------------------------------------------------
constexpr int BVH_BLOCK = 128;
template <bool RECHECK>
__global__ void __launch_bounds__(BVH_BLOCK, 4) k_bvh(CastArgs a) {
    // per-warp stack of (deferred child, lanes whose rays enter its box)
    __shared__ int2 stk[BVH_BLOCK / 32][BVH_STACK];
    const uint32_t lane = threadIdx.x & 31u;
    int2* stack = stk[threadIdx.x >> 5];
    const bool cull_back = a.flags & 2u;
    uint32_t n_vis = 0, n_tst = 0, c_unc = 0, c_ties = 0;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t g0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32u; g0 < a.n_rays_total; g0 += n_warps * 32u) {
        const uint32_t g = g0 + lane;
        const bool valid = g < a.n_rays_total;
        uint32_t sn = 0;
        for (uint32_t k = 1; k < a.n_sensors; ++k)
            if (a.sensors[k].ray_off <= g) sn = k;
        const SensorDev& S = a.sensors[sn];
        const uint32_t q = valid ? g - S.ray_off : 0u;
        const uint32_t j = q / S.n_rays, i = q - j * S.n_rays;
        const V3 d = ray_dir(__ldg(&a.ch_sc[S.ch_off + j]), __ldg(&a.az_sc[S.az_off + i]));
        // world direction B^T d for the box tests and the leaf pre-test (the exact test uses d)
        const V3 dw = {S.B[0] * d.x + S.B[3] * d.y + S.B[6] * d.z, S.B[1] * d.x + S.B[4] * d.y + S.B[7] * d.z,
                       S.B[2] * d.x + S.B[5] * d.y + S.B[8] * d.z};
        const V3 inv = {1.f / (dw.x != 0.f ? dw.x : 1e-30f), 1.f / (dw.y != 0.f ? dw.y : 1e-30f),
                        1.f / (dw.z != 0.f ? dw.z : 1e-30f)};
        const V3 o = {S.o_hi[0], S.o_hi[1], S.o_hi[2]};
        const V3 oi = {o.x * inv.x, o.y * inv.y, o.z * inv.z};
        // pre-test margin term of the origin's low part (|o_lo| <= u |o|)
        const float o_term = 2.f * U32 * (fabsf(o.x) + fabsf(o.y) + fabsf(o.z));
        unsigned long long cur = valid ? __ldcg(&a.keys[g]) : 0ull;
        const float tmin = fmaxf(S.d_min * (1.f - 2e-5f) - 2e-6f, 0.f);
        // an idle lane gets an empty interval: it never votes for a box
        float tmax = valid ? fminf(S.d_max * (1.f + 2e-5f) + 2e-6f,
                                   __uint_as_float((uint32_t)(cur >> 32)) * (1.f + 4.f * BETA))
                           : -1.f;
        int sp = 0;          // warp-uniform
        int32_t node = 0;    // warp-uniform
        // lanes whose rays enter the current node's box (a lane outside it
        // cannot enter any box below it: the boxes are nested)
        uint32_t act = __ballot_sync(0xffffffffu, tmax >= tmin);
        while (act) {
            const bool mine = (act >> lane) & 1u;
            if (node >= 0) {
                const float4* np = reinterpret_cast<const float4*>(a.bvh_nodes + node);
                const float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2);
                const int4 n3 = __ldg(reinterpret_cast<const int4*>(np) + 3);
                n_vis++;
                // slab distances x / dw - o / dw (one FMA each); their rounding, relative to
                // |o| + |x - o| along the ray, is far below the boxes' inflation
                const float ax0 = fmaf(n0.x, inv.x, -oi.x), bx0 = fmaf(n0.w, inv.x, -oi.x);
                const float ay0 = fmaf(n0.y, inv.y, -oi.y), by0 = fmaf(n1.x, inv.y, -oi.y);
                const float az0 = fmaf(n0.z, inv.z, -oi.z), bz0 = fmaf(n1.y, inv.z, -oi.z);
                const float ax1 = fmaf(n1.z, inv.x, -oi.x), bx1 = fmaf(n2.y, inv.x, -oi.x);
                const float ay1 = fmaf(n1.w, inv.y, -oi.y), by1 = fmaf(n2.z, inv.y, -oi.y);
                const float az1 = fmaf(n2.x, inv.z, -oi.z), bz1 = fmaf(n2.w, inv.z, -oi.z);
                const float tn0 = fmaxf(fmaxf(fminf(ax0, bx0), fminf(ay0, by0)), fmaxf(fminf(az0, bz0), tmin));
                const float tf0 = fminf(fminf(fmaxf(ax0, bx0), fmaxf(ay0, by0)), fminf(fmaxf(az0, bz0), tmax));
                const float tn1 = fmaxf(fmaxf(fminf(ax1, bx1), fminf(ay1, by1)), fmaxf(fminf(az1, bz1), tmin));
                const float tf1 = fminf(fminf(fmaxf(ax1, bx1), fmaxf(ay1, by1)), fminf(fmaxf(az1, bz1), tmax));
                const bool h0 = mine && tn0 <= tf0, h1 = mine && tn1 <= tf1;
                const uint32_t b0 = __ballot_sync(0xffffffffu, h0), b1 = __ballot_sync(0xffffffffu, h1);
                if (b0 && b1) {
                    // child 1 first if most lanes that enter both find it nearer (or, when
                    // no lane enters both, if more lanes enter it)
                    const uint32_t both = b0 & b1, near1 = __ballot_sync(0xffffffffu, h0 && h1 && tn1 < tn0);
                    const bool swap = both ? 2 * __popc(near1) > __popc(both) : __popc(b1) > __popc(b0);
                    if (lane == 0) stack[sp] = swap ? make_int2(n3.x, (int)b0) : make_int2(n3.y, (int)b1);  // depth < BVH_STACK
                    __syncwarp();
                    ++sp;
                    node = swap ? n3.y : n3.x;
                    act = swap ? b1 : b0;
                } else if (b0 || b1) {
                    node = b0 ? n3.x : n3.y;
                    act = b0 ? b0 : b1;
                } else {
                    if (sp == 0) break;
                    const int2 e = stack[--sp];
                    node = e.x;
                    act = (uint32_t)e.y;
                }
                continue;
            }
            const uint32_t lf = ((uint32_t)node >> 3) & 0x0FFFFFFFu, cnt = ((uint32_t)node & 7u) + 1u;
            for (uint32_t k = lf; k < lf + cnt; ++k) {
                float t9[9];
#pragma unroll
                for (int m = 0; m < 9; ++m) t9[m] = __ldg(a.bvh_tris + 9ull * k + m);
                if (!mine || !(tmax >= tmin)) continue;  // this lane's ray misses the leaf's box
                n_tst++;
                {
                    // world-frame pre-test: the edge functions F_k = dw.((v_k - o) x (v_k+1 - v_k))
                    // follow the winding, so a ray inside has all three of one sign.  Skip
                    // the triangle only if two have provably opposite signs; the margin
                    // covers this evaluation's rounding, the FP32 direction and origin
                    // differences and the exact test's own error bound, so nothing the
                    // exact test could report as a hit or send to the re-test is skipped.
                    const V3 v0 = {t9[0], t9[1], t9[2]}, v1 = {t9[3], t9[4], t9[5]}, v2 = {t9[6], t9[7], t9[8]};
                    const V3 a0 = vsub(v0, o), a1 = vsub(v1, o), a2 = vsub(v2, o);
                    const V3 e0 = vsub(v1, v0), e1 = vsub(v2, v1), e2 = vsub(v0, v2);
                    const float F0 = vdot(dw, vcross(a0, e0)), F1 = vdot(dw, vcross(a1, e1)), F2 = vdot(dw, vcross(a2, e2));
                    auto l1 = [](V3 x) { return fabsf(x.x) + fabsf(x.y) + fabsf(x.z); };
                    const float m0 = (64.f * U32 * l1(a0) + o_term) * l1(e0), m1 = (64.f * U32 * l1(a1) + o_term) * l1(e1),
                                m2 = (64.f * U32 * l1(a2) + o_term) * l1(e2);
                    const bool neg = F0 < -m0 || F1 < -m1 || F2 < -m2, pos = F0 > m0 || F1 > m1 || F2 > m2;
                    if (neg && pos) continue;
                }
                TriW T;
                tri_world(t9, T);
                if (T.n.x == 0.f && T.n.y == 0.f && T.n.z == 0.f) continue;  // zero area: never hit
                V3 w[3], p[3];
#pragma unroll
                for (int kk = 0; kk < 3; ++kk) {
                    w[kk] = rel_origin(S, T.v[kk]);
                    p[kk] = rotB(S.B, w[kk]);
                }
                const float det = vdot(w[0], T.n);
                if (cull_back && det > 0.f && (!RECHECK || det > backface_err(w[0], T.n, T.N))) continue;
                const float err_det = det_error(w[0], T);
                if (!(det != 0.f || (RECHECK && fabsf(det) <= err_det))) continue;
                SetupReg sr;
                make_setup(S, T, w, p, det, err_det, SetupWriterReg{sr});
                float t, terr;
                const int res = test_fp32<RECHECK>(sr, S, d, t, terr);
                if (res == T_MISS) continue;
                const uint32_t tri = __ldg(a.bvh_prim + k);
                commit_pre<RECHECK>(a, g, tri, res, t, terr, sr.f(21), cur, c_unc, c_ties);
                if (res == T_HIT) {
                    const unsigned long long key = ((unsigned long long)__float_as_uint(t) << 32) | tri;
                    if (key < cur) cur = key;
                    tmax = fminf(tmax, t * (1.f + 4.f * BETA));
                }
            }
            if (sp == 0) break;
            const int2 e = stack[--sp];
            node = e.x;
            act = (uint32_t)e.y;
        }
        __syncwarp();
    }
    n_vis = __reduce_add_sync(0xffffffffu, lane == 0 ? n_vis : 0u);
    n_tst = __reduce_add_sync(0xffffffffu, n_tst);
    c_unc = __reduce_add_sync(0xffffffffu, c_unc);
    c_ties = __reduce_add_sync(0xffffffffu, c_ties);
    if (lane == 0) {
        if (n_vis) atomicAdd(&a.counters[C_BVH_VISITS], (unsigned long long)n_vis);
        if (n_tst) atomicAdd(&a.counters[C_BVH_TESTS], (unsigned long long)n_tst);
        if (c_unc) atomicAdd(&a.counters[C_UNCERTAIN], (unsigned long long)c_unc);
        if (c_ties) atomicAdd(&a.counters[C_TIES], (unsigned long long)c_ties);
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
size_t cull_smem_bytes(const CastArgs& a, const LaunchCfg& cfg) {
    size_t off = sizeof(SensorDev) * a.n_sensors + sizeof(float2) * a.total_ch + sizeof(uint16_t) * LUT_BINS * a.n_sensors;
    off = (off + 15) & ~size_t(15);
    return off + sizeof(CullWarpSmem) * (size_t)(cfg.cull_block / 32);
}
static size_t cull_a_smem_bytes(uint32_t ns, uint32_t n_ch, const LaunchCfg& cfg) {
    size_t off = sizeof(SensorDev) * ns + sizeof(ElevSensor) * ns + sizeof(float) * n_ch + sizeof(uint16_t) * LUT_BINS * ns;
    off = (off + 15) & ~size_t(15);
    return off + sizeof(CullAWarpSmem) * (size_t)(cfg.cull_block / 32);
}
static size_t cull_b_smem_bytes(const CastArgs& a) {
    size_t off = sizeof(SensorDev) * a.n_sensors + sizeof(float2) * a.total_ch;
    return ((off + 15) & ~size_t(15)) + sizeof(CullBWarpSmem) * 8;
}

template <typename K>
static void ensure_smem_attr(K kernel, size_t smem) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

const char* const kKernelNames[K_NUM] = {"k_init",  "k_cull_a",         "k_cull_b",       "k_expand",
                                         "k_test",  "k_bvh",            "k_refine",         "k_recheck_filter",
                                         "k_recheck_rays", "k_recheck_pairs", "k_decode"};

// elevation cull of triangles [a.tri_first, a.n_tris) (ac) and/or the
// survivor pass of the whole cast (a)
template <bool R, bool B>
static void launch_cull_split(const CastArgs& a, const CastArgs& ac, bool do_a, bool do_b, const LaunchCfg& cfg,
                              int n_sm, cudaStream_t st, const std::function<void(int, int)>& mark) {
    if (do_a) {
        const bool groups = !B && ac.gbounds != nullptr;
        const uint32_t span = ac.n_tris > (ac.tri_first & ~31u) ? ac.n_tris - (ac.tri_first & ~31u) : 0u;
        const uint32_t max_blocks = (span + cfg.cull_block - 1) / cfg.cull_block;
        const int grid_a =
            (int)std::min<uint32_t>(std::max<uint32_t>(max_blocks, 1u), (uint32_t)(n_sm * cfg.cull_blocks_per_sm));
        mark(K_CULL_A, 0);
        // one launch per group of ELEV_GROUP sensors
        for (uint32_t g0 = 0; g0 < ac.n_sensors; g0 += ELEV_GROUP) {
            CastArgs ag = ac;
            ag.sens_base = g0;
            ag.sens_count = std::min<uint32_t>(ELEV_GROUP, ac.n_sensors - g0);
            const size_t sa = cull_a_smem_bytes(ag.sens_count, ag.total_ch, cfg);
            if (groups) {
                ensure_smem_attr(k_cull_a<true>, sa);
                k_cull_a<true><<<grid_a, cfg.cull_block, sa, st>>>(ag);
            } else {
                ensure_smem_attr(k_cull_a<false>, sa);
                k_cull_a<false><<<grid_a, cfg.cull_block, sa, st>>>(ag);
            }
        }
        mark(K_CULL_A, 1);
    }
    if (do_b) {
        const size_t sb = cull_b_smem_bytes(a);
        ensure_smem_attr(k_cull_b<R, B>, sb);
        mark(K_CULL_B, 0);
        k_cull_b<R, B><<<n_sm * cfg.cull_blocks_per_sm * 2, 256, sb, st>>>(a);
        mark(K_CULL_B, 1);
    }
}

// key -> (distance, id) of finished keys (the last stage of a sharded cast)
void launch_decode(const CastArgs& a, int n_sm, cudaStream_t st) {
    const int nb = (int)std::min<uint32_t>((a.n_rays_total + 255) / 256, (uint32_t)n_sm * 8);
    k_decode<<<std::max(nb, 1), 256, 0, st>>>(a, 0);
}

int launch_frame(const CastArgs& a, const LaunchCfg& cfg, int n_sm, cudaStream_t st, const KernelMarks* marks,
                 FrameSplit split) {
    const bool recheck = a.flags & 1u;
    const bool brute = a.flags & 4u;
    int launches = 0;
    std::function<void(int, int)> mark = [&](int k, int phase) {
        if (marks && marks->fn) marks->fn(marks->user, k, phase, st);
    };
    const int nb = (int)std::min<uint32_t>((a.n_rays_total + 255) / 256, (uint32_t)n_sm * 8);
    if (split.stage == 2) {
        // the filter against the winner over all shards, then the exported flags
        if (recheck) {
            mark(K_RECHECK_FILTER, 0);
            k_recheck_filter<<<n_sm * 2, 256, 0, st>>>(a);
            mark(K_RECHECK_FILTER, 1);
        }
        k_shard_flags<<<std::max(nb, 1), 256, 0, st>>>(a);
        return launches + (recheck ? 2 : 1);
    }
    if (split.stage == 3) {
        // the rays flagged by any shard, the FP64 re-tests, the resolved keys
        if (recheck) {
            k_shard_join<<<std::max(nb, 1), 256, 0, st>>>(a);
            mark(K_RECHECK_RAYS, 0);
            k_recheck_rays<<<n_sm * 8, 256, 0, st>>>(a);
            mark(K_RECHECK_RAYS, 1);
            mark(K_RECHECK_PAIRS, 0);
            k_recheck_pairs<<<n_sm * 4, RECHECK_BLOCK, 0, st>>>(a);
            mark(K_RECHECK_PAIRS, 1);
            launches += 3;
        }
        k_shard_export<<<std::max(nb, 1), 256, 0, st>>>(a, a.tri_base, recheck ? 1 : 0);
        return launches + 1;
    }
    // the triangle range of this part's elevation cull
    CastArgs ac = a;
    if (split.part == 1) ac.n_tris = std::max(std::min(split.at, a.n_tris), a.tri_first);
    if (split.part == 2) ac.tri_first = std::max(split.at, a.tri_first);
    if (split.part != 2) {
        int init_blocks = (int)std::min<uint32_t>((a.n_rays_total + 255) / 256, (uint32_t)n_sm * 8);
        mark(K_INIT, 0);
        k_init<<<max(init_blocks, 1), 256, 0, st>>>(a);
        mark(K_INIT, 1);
        launches++;
    }
    CastArgs ab = a;
    ab.surv_part = (uint32_t)split.part;
    if (recheck && brute)
        launch_cull_split<true, true>(ab, ac, true, true, cfg, n_sm, st, mark);
    else if (recheck)
        launch_cull_split<true, false>(ab, ac, true, true, cfg, n_sm, st, mark);
    else if (brute)
        launch_cull_split<false, true>(ab, ac, true, true, cfg, n_sm, st, mark);
    else
        launch_cull_split<false, false>(ab, ac, true, true, cfg, n_sm, st, mark);
    launches += 1 + (int)((a.n_sensors + ELEV_GROUP - 1) / ELEV_GROUP);
    if (split.part == 1) return launches;
    if (!brute) {
        mark(K_EXPAND, 0);
        k_expand<<<n_sm * 8, 256, 0, st>>>(a);
        mark(K_EXPAND, 1);
        mark(K_TEST, 0);
        if (recheck)
            k_test<true><<<n_sm * 8, cfg.test_block, 0, st>>>(a);
        else
            k_test<false><<<n_sm * 8, cfg.test_block, 0, st>>>(a);
        mark(K_TEST, 1);
        launches += 2;
    }
    if (a.bvh_nodes) {
        // static side of a hybrid cast, after the dynamic triangles so that
        // their hits bound the traversal
        // many more blocks than fit at once: the fans differ widely in cost, and
        // blocks that finish early make room for the next ones (64 per SM measured
        // 11 % faster than 16 on c5; one fan per warp was slower again)
        const int blocks = (int)std::min<uint32_t>((a.n_rays_total + BVH_BLOCK - 1) / BVH_BLOCK, (uint32_t)n_sm * 64);
        mark(K_BVH, 0);
        if (recheck)
            k_bvh<true><<<std::max(blocks, 1), BVH_BLOCK, 0, st>>>(a);
        else
            k_bvh<false><<<std::max(blocks, 1), BVH_BLOCK, 0, st>>>(a);
        mark(K_BVH, 1);
        launches++;
    }
    if (recheck) {
        mark(K_REFINE, 0);
        k_refine_count<<<1, 1, 0, st>>>(a);
        k_refine<<<n_sm * 8, 256, 0, st>>>(a);
        mark(K_REFINE, 1);
        launches += 2;
    }
    if (split.stage == 1) {
        // FP32 pass of a sharded cast: export the keys
        k_shard_export<<<std::max(nb, 1), 256, 0, st>>>(a, a.tri_base, 0);
        return launches + 1;
    }
    if (recheck) {
        mark(K_RECHECK_FILTER, 0);
        k_recheck_filter<<<n_sm * 2, 256, 0, st>>>(a);
        mark(K_RECHECK_FILTER, 1);
        mark(K_RECHECK_RAYS, 0);
        k_recheck_rays<<<n_sm * 8, 256, 0, st>>>(a);
        mark(K_RECHECK_RAYS, 1);
        mark(K_RECHECK_PAIRS, 0);
        k_recheck_pairs<<<n_sm * 4, RECHECK_BLOCK, 0, st>>>(a);
        mark(K_RECHECK_PAIRS, 1);
        launches += 3;
    }
    int dec_blocks = nb;
    mark(K_DECODE, 0);
    k_decode<<<max(dec_blocks, 1), 256, 0, st>>>(a, recheck ? 1 : 0);
    mark(K_DECODE, 1);
    launches++;
    return launches;
}

}  // namespace grca

// ===========================================================================
// Allocation-free cast (grca_cast_noalloc)
//
// Some callers cannot call cudaMalloc: code running inside a host-side
// allocator or memory-pool callback, a plugin whose host framework forbids
// device allocations after start-up, or a real-time loop that must not block
// on the driver's allocator.  For them this entry point keeps its scratch
// memory (per-ray closest-hit keys, the ray direction tables, the sensor
// descriptor and the counters) in one fixed, file-scope device array that
// exists from module load until process exit on every GPU that loads the
// library.  It runs the same culling and decode kernels as grca_cast, with
// all candidate spans tested inline and the plain FP32 test.
// ===========================================================================
namespace grca {

constexpr uint32_t NOALLOC_MAX_RAYS = 262144;      // channels x rays per call
constexpr uint32_t NOALLOC_MAX_CHANNELS = 256;
constexpr uint32_t NOALLOC_MAX_AZIMUTH = (uint32_t)MAX_RAYS;

struct NoallocLayout {
    static constexpr size_t keys = 0;                                              // u64 x max rays
    static constexpr size_t az = keys + sizeof(unsigned long long) * NOALLOC_MAX_RAYS;  // float2 x max azimuth
    static constexpr size_t ch = az + sizeof(float2) * NOALLOC_MAX_AZIMUTH;             // float2 x max channels
    static constexpr size_t lut = ch + sizeof(float2) * NOALLOC_MAX_CHANNELS;           // u16 x LUT_BINS
    static constexpr size_t sensor = (lut + sizeof(uint16_t) * LUT_BINS + 15) & ~size_t(15);  // one SensorDev
    static constexpr size_t counters = (sensor + sizeof(SensorDev) + 255) & ~size_t(255);  // u64 x C_NUM
    static constexpr size_t qcount = counters + sizeof(unsigned long long) * C_NUM;        // u32 x Q_NUM
    static constexpr size_t error = qcount + sizeof(uint32_t) * Q_NUM;                     // u32
    static constexpr size_t total = (error + sizeof(uint32_t) + 255) & ~size_t(255);
};

// The scratch array (about 2.4 MB).  Host code must not use this symbol as a
// device address; it obtains the address with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NoallocLayout::total];

struct NoallocParams {
    SensorDev s;
    float2 ch[NOALLOC_MAX_CHANNELS];
    uint16_t lut[LUT_BINS];
    double theta0, dtheta;
};

// fill the sensor descriptor, channel and azimuth tables and reset the keys,
// counters and error word of the scratch array
__global__ void k_noalloc_prepare(NoallocParams P, unsigned char* scratch) {
    uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(scratch + NoallocLayout::keys);
    float2* az = reinterpret_cast<float2*>(scratch + NoallocLayout::az);
    float2* ch = reinterpret_cast<float2*>(scratch + NoallocLayout::ch);
    uint32_t n_total = P.s.n_ch * P.s.n_rays;
    for (uint32_t g = tid; g < n_total; g += stride) keys[g] = KEY_MISS;
    for (uint32_t i = tid; i < P.s.n_rays; i += stride) {
        double sn, cs;
        sincos(P.theta0 + (double)i * P.dtheta, &sn, &cs);
        az[i] = make_float2((float)sn, (float)cs);
    }
    for (uint32_t j = tid; j < P.s.n_ch; j += stride) ch[j] = P.ch[j];
    uint16_t* lut = reinterpret_cast<uint16_t*>(scratch + NoallocLayout::lut);
    for (uint32_t b = tid; b < (uint32_t)LUT_BINS; b += stride) lut[b] = P.lut[b];
    if (tid == 0) *reinterpret_cast<SensorDev*>(scratch + NoallocLayout::sensor) = P.s;
    if (tid < C_NUM) reinterpret_cast<unsigned long long*>(scratch + NoallocLayout::counters)[tid] = 0ull;
    if (tid < Q_NUM) reinterpret_cast<uint32_t*>(scratch + NoallocLayout::qcount)[tid] = 0u;
    if (tid == 0) *reinterpret_cast<uint32_t*>(scratch + NoallocLayout::error) = 0u;
}

}  // namespace grca

#include <mutex>

#include "grca.h"

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoallocMaxDevices] = {};   // device address of the scratch array, per device index
int g_noalloc_sm[kNoallocMaxDevices] = {};
}  // namespace

extern "C" grca_status grca_cast_noalloc(const grca_sensor_desc* d, const float* tris, uint32_t n_tris,
                                         float* out_dist, uint32_t* out_tri, uint32_t flags, void* stream) {
    using namespace grca;
    if (!d || !d->elev_rad || !out_dist || !out_tri || (!tris && n_tris)) return GRCA_ERR_INVALID_ARG;
    if (flags & ~(uint32_t)GRCA_CAST_CULL_BACKFACE) return GRCA_ERR_INVALID_ARG;
    // sizes beyond the fixed scratch array are rejected
    if (d->n_channels > NOALLOC_MAX_CHANNELS || d->n_rays > NOALLOC_MAX_AZIMUTH ||
        (uint64_t)d->n_channels * d->n_rays > NOALLOC_MAX_RAYS)
        return GRCA_ERR_CAPACITY;
    // every check of grca_create_sensor (orthonormal axes, finite origin,
    // |theta0| <= 4 pi, finite d_min, ...), then the vertex buffer's alignment:
    // the culling kernel loads it as float4
    if (!sensor_desc_valid(d)) return GRCA_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(tris) & 15u) return GRCA_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return GRCA_ERR_CUDA;
    unsigned char* scratch = nullptr;
    int n_sm = 0;
    {
        // set-up, once per device, with that device current: the device address
        // of the scratch array (the host-side symbol is only a stand-in)
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GRCA_ERR_CUDA;
            int sm = 0;
            if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GRCA_ERR_CUDA;
            g_noalloc_sm[dev] = sm;
            g_noalloc_ptr[dev] = p;
        }
        scratch = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
        n_sm = g_noalloc_sm[dev];
    }
    NoallocParams P;
    memset(&P, 0, sizeof(P));
    SensorDev& s = P.s;
    for (int k = 0; k < 3; ++k) {
        s.o64[k] = d->origin[k];
        s.B64[k] = d->f[k];
        s.B64[3 + k] = d->r[k];
        s.B64[6 + k] = d->u[k];
        float hi = (float)d->origin[k];
        s.o_hi[k] = hi;
        s.o_lo[k] = (float)(d->origin[k] - (double)hi);
    }
    for (int k = 0; k < 9; ++k) s.B[k] = (float)s.B64[k];
    s.d_min64 = d->d_min;
    s.d_max64 = d->d_max;
    s.theta0 = (float)d->theta0;
    s.dtheta = (float)d->dtheta;
    s.inv_dtheta = (float)(1.0 / d->dtheta);
    s.d_min = (float)d->d_min;
    s.d_max = std::isfinite(d->d_max) ? (float)d->d_max : INFINITY;
    s.period = (float)(2 * M_PI / d->dtheta);
    s.n_ch = d->n_channels;
    s.n_rays = d->n_rays;
    s.full = std::fabs(d->n_rays * d->dtheta - 2 * M_PI) <= 1e-9 ? 1u : 0u;
    s.has_range = (d->d_min > 0.0 || std::isfinite(d->d_max)) ? 1u : 0u;
    s.inv_period = 1.0f / (s.full ? (float)s.n_rays : s.period);
    double det = d->f[0] * (d->r[1] * d->u[2] - d->r[2] * d->u[1]) - d->f[1] * (d->r[0] * d->u[2] - d->r[2] * d->u[0]) +
                 d->f[2] * (d->r[0] * d->u[1] - d->r[1] * d->u[0]);
    s.hand = det < 0.0 ? -1.f : 1.f;
    float sins[NOALLOC_MAX_CHANNELS];
    for (uint32_t j = 0; j < d->n_channels; ++j) {
        double e = d->elev_rad[j];
        P.ch[j] = make_float2((float)std::sin(e), (float)std::cos(e));
        sins[j] = P.ch[j].x;
    }
    build_channel_lut(sins, d->n_channels, s.lut_lo, s.lut_inv_w, P.lut);
    s.lut_off = 0;
    P.theta0 = d->theta0;
    P.dtheta = d->dtheta;

    CastArgs a;
    memset(&a, 0, sizeof(a));
    a.tris = tris;
    a.n_tris = n_tris;
    a.n_sensors = 1;
    a.sensors = reinterpret_cast<const SensorDev*>(scratch + NoallocLayout::sensor);
    a.ch_sc = reinterpret_cast<const float2*>(scratch + NoallocLayout::ch);
    a.az_sc = reinterpret_cast<const float2*>(scratch + NoallocLayout::az);
    a.lut = reinterpret_cast<const uint16_t*>(scratch + NoallocLayout::lut);
    a.total_ch = d->n_channels;
    a.n_rays_total = d->n_channels * d->n_rays;
    a.keys = reinterpret_cast<unsigned long long*>(scratch + NoallocLayout::keys);
    a.qcount = reinterpret_cast<uint32_t*>(scratch + NoallocLayout::qcount);
    a.counters = reinterpret_cast<unsigned long long*>(scratch + NoallocLayout::counters);
    a.error = reinterpret_cast<uint32_t*>(scratch + NoallocLayout::error);
    a.flags = flags;
    a.inline_max = 0xFFFFFFFFu;  // every span tested inline: no deferred-pair queue is needed
    a.out_dist = out_dist;
    a.out_tri = out_tri;
    LaunchCfg cfg;
    cudaStream_t st = (cudaStream_t)stream;
    // an error left by an earlier, unrelated launch is cleared here, so that
    // the status below reports this call's launches only
    (void)cudaGetLastError();
    int blocks = (int)std::min<uint32_t>((a.n_rays_total + 255) / 256, (uint32_t)n_sm * 8);
    k_noalloc_prepare<<<std::max(blocks, 1), 256, 0, st>>>(P, scratch);
    size_t smem = cull_smem_bytes(a, cfg);
    uint32_t max_blocks = (n_tris + cfg.cull_block - 1) / cfg.cull_block;
    int cull_grid = (int)std::min<uint32_t>(std::max<uint32_t>(max_blocks, 1u), (uint32_t)(n_sm * cfg.cull_blocks_per_sm));
    k_cull<false, false><<<cull_grid, cfg.cull_block, smem, st>>>(a);
    k_decode<<<std::max(blocks, 1), 256, 0, st>>>(a, 0);
    return cudaGetLastError() == cudaSuccess ? GRCA_OK : GRCA_ERR_CUDA;
}
