/* GRCA CPU oracle: plain FP64 brute force over all rays x all triangles.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header or table with the CUDA path.
 *
 * What it computes (the problem statement of Sec. 1.1, Eq. brute): for every
 * ray of every spinning LiDAR, the closest triangle that the ray intersects
 * and its distance.  Rays follow Eq. ray_dir (Sec. 3.1):
 *     d = cos(theta) cos(phi) f + sin(theta) cos(phi) r + sin(phi) u,
 *     theta = theta0 + i*dtheta,  phi = elev[j];
 * the ray is o + t d, t > 0.  A triangle (closed: edges and vertices
 * included) is hit at t when o + t d lies in it; zero-area triangles and rays
 * parallel to the plane never hit.  A hit counts only if d_min <= t <= d_max
 * (per-hit reading of the range filter of App. A.4.1).  With back-face
 * culling on, only triangles whose normal n = (v1-v0)x(v2-v0) satisfies
 * n.(o - v0) > 0 count.  Closest = smallest t, ties to the lower id (the
 * paper keeps only the minimum distance, Sec. A.5.2).  A miss reports
 * t = +inf and id = 0xFFFFFFFF (Sec. A.5.1).
 *
 * Global ray ids follow the global ray index of App. A.4.1 (Step 5):
 * g = O_n + j * n_rays_n + i (sensor-major, then channel, then ray).
 */
#ifndef GRCA_ORACLE_H
#define GRCA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_TIES 16
#define ORC_NO_HIT 0xFFFFFFFFu

typedef struct {
    double origin[3];
    double f[3], r[3], u[3];   /* forward, right, up (orthonormal) */
    double theta0, dtheta;     /* azimuth grid */
    double d_min, d_max;       /* range; d_max may be +inf */
    const double* elev;        /* n_channels elevations (radians) */
    uint32_t n_channels;
    uint32_t n_rays;
    const double* theta;       /* nullable: n_rays per-ray azimuths replacing theta0 + i*dtheta
                                  (horizontal noise, App. A.1) */
    const uint32_t* mask;      /* nullable: ray (j, i) fires iff bit q & 31 of mask[q >> 5] is set,
                                  q = j*n_rays + i (ray-mask images, App. A.3); a ray that does
                                  not fire is a miss */
} orc_sensor;

/* Ray direction of (channel j, ray i): Eq. ray_dir, with theta[i] in place
 * of theta0 + i*dtheta when the sensor has per-ray azimuths. */
void orc_ray_dir(const orc_sensor* s, uint32_t j, uint32_t i, double d[3]);

/* One ray against one triangle (9 floats: v0, v1, v2).  Returns 1 and *t on
 * a hit with t > 0 (no range or facing test here). */
int orc_hit(const double o[3], const double d[3], const float* tri, double* t);

/* Facing rule: 1 if n.(o - v0) > 0 with n = (v1-v0)x(v2-v0). */
int orc_faces(const double o[3], const float* tri);

/* Brute force over the listed global ray ids.
 *   best_t/best_id    : closest hit (+inf / 0xFFFFFFFF on a miss)
 *   second_t          : (nullable) smallest t among hits of triangles other than best_id
 *   n_ties, tie_ids   : (nullable) triangles with t <= best_t*(1+tie_rel);
 *                       up to ORC_MAX_TIES ids per ray, ascending id
 *   n_tests           : (nullable) number of ray-triangle tests run (Eq. brute)
 * Returns 0, or -1 on a bad ray id / argument. */
int orc_cast(const orc_sensor* sensors, uint32_t n_sensors,
             const float* tris, uint32_t n_tris,
             const int64_t* ray_ids, int64_t n_rays,
             int cull_backface, double tie_rel, int n_threads,
             double* best_t, uint32_t* best_id,
             double* second_t, uint32_t* n_ties, uint32_t* tie_ids,
             uint64_t* n_tests, const uint8_t* keep);
/* keep (nullable): n_sensors x n_tris bytes; triangle k is ignored for the
 * rays of sensor n when keep[n * n_tris + k] == 0. */

/* Apparent-area filter of App. A.4.1 Step 1 (Eq. apparent_area): for every
 * (sensor n, triangle k), with A_T the area, c the centroid and n^ the unit
 * normal, the pair is dropped when (A_T (c-o).n^)^2 < eps^2 |c-o|^6.
 * out[n * n_tris + k] = 1 keep, 0 drop, 2 keep but within a relative 1e-3 of
 * the threshold (where an FP32 evaluation may decide either way). */
void orc_area_keep(const orc_sensor* sensors, uint32_t n_sensors, const float* tris, uint32_t n_tris, double eps,
                   uint8_t* out);

/* Range noise (App. A.1: added to the distance after output conversion):
 * z[k] = sqrt(-2 ln u1) cos(2 pi u2), the Box-Muller transform (Box and
 * Muller, 1958) of u1 = (top24(a) + 1) / 2^24 and u2 = top24(b) / 2^24, where
 * a = sm(seed + 2 q[k]), b = sm(seed + 2 q[k] + 1) and sm(x) is the SplitMix64
 * output for state x (Steele, Lea and Flood, 2014): x + 0x9E3779B97F4A7C15,
 * then the two xor-shift-multiply rounds and a final xor-shift.  q is the
 * ray's index j*n_rays + i within its sensor.  Arithmetic in FP64. */
void orc_range_noise(uint64_t seed, const int64_t* q, int64_t n, double* z);

/* The SplitMix64 output function sm(x) above (exposed for its published test vectors). */
uint64_t orc_splitmix64(uint64_t x);

/* Grading helper for one (ray, triangle): t of the ray with the triangle's
 * plane (+inf if parallel or degenerate) and the signed angular margin of the
 * ray w.r.t. the triangle seen from o: min over edges of asin(s_k d.m_k),
 * m_k the unit normal of the plane through o and edge k, s_k orienting the
 * triangle's interior positive.  margin >= 0 means inside (for t > 0). */
int orc_ray_tri_margin(const orc_sensor* sensors, uint32_t n_sensors, int64_t ray_id,
                       const float* tri, double* t_plane, double* margin);

/* Every ray of sensor `sensor` that hits triangle k (two-sided, in range):
 * writes (k_local, local ray id j*n_rays+i) pairs for tris[0..n_tris) into
 * out[2*m], up to cap pairs.  Returns the total number of pairs (may exceed cap). */
int64_t orc_triangle_hits(const orc_sensor* sensor, const float* tris, uint32_t n_tris,
                          int cull_backface, int n_threads, int64_t* out, int64_t cap);

#ifdef __cplusplus
}
#endif
#endif
