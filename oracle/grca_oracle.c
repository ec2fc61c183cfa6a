/* GRCA CPU oracle: plain FP64 brute force (TEST INFRASTRUCTURE ONLY).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this library.  It shares no code with the CUDA path.  Every function below
 * follows the problem statement (Sec. 1.1, Eq. brute), the ray formula
 * (Sec. 3.1, Eq. ray_dir) and the output convention (Sec. A.5.1); see
 * grca_oracle.h for the exact definition of the result.
 *
 * The ray-triangle test is the textbook one, written out: intersect the ray
 * with the triangle's plane, then check that the point lies on the inner side
 * of all three edges.  It is deliberately not the formulation the GPU uses.
 */
#include "grca_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

static void sub3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}
static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static void load_tri(const float* tri, double v0[3], double v1[3], double v2[3]) {
    for (int k = 0; k < 3; ++k) {
        v0[k] = (double)tri[k];
        v1[k] = (double)tri[3 + k];
        v2[k] = (double)tri[6 + k];
    }
}

/* Eq. ray_dir (Sec. 3.1): d = cos(th)cos(ph) f + sin(th)cos(ph) r + sin(ph) u;
 * th is the ray's own azimuth when the sensor lists perturbed ones (App. A.1). */
void orc_ray_dir(const orc_sensor* s, uint32_t j, uint32_t i, double d[3]) {
    double th = s->theta ? s->theta[i] : s->theta0 + (double)i * s->dtheta;
    double ph = s->elev[j];
    double a = cos(th) * cos(ph), b = sin(th) * cos(ph), c = sin(ph);
    for (int k = 0; k < 3; ++k) d[k] = a * s->f[k] + b * s->r[k] + c * s->u[k];
}

/* Plane intersection, then the three same-side tests (closed triangle). */
int orc_hit(const double o[3], const double d[3], const float* tri, double* t_out) {
    double v0[3], v1[3], v2[3], e1[3], e2[3], n[3], w[3], x[3];
    load_tri(tri, v0, v1, v2);
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(e1, e2, n);
    if (dot3(n, n) == 0.0) return 0;          /* zero-area triangle */
    double denom = dot3(n, d);
    if (denom == 0.0) return 0;               /* ray parallel to the plane */
    sub3(v0, o, w);
    double t = dot3(n, w) / denom;
    if (!(t > 0.0)) return 0;                 /* plane behind the origin */
    for (int k = 0; k < 3; ++k) x[k] = o[k] + t * d[k];
    const double* V[3] = {v0, v1, v2};
    for (int k = 0; k < 3; ++k) {
        const double* a = V[k];
        const double* b = V[(k + 1) % 3];
        double ab[3], ax[3], c[3];
        sub3(b, a, ab);
        sub3(x, a, ax);
        cross3(ab, ax, c);
        if (dot3(c, n) < 0.0) return 0;       /* outside edge k */
    }
    *t_out = t;
    return 1;
}

int orc_faces(const double o[3], const float* tri) {
    double v0[3], v1[3], v2[3], e1[3], e2[3], n[3], w[3];
    load_tri(tri, v0, v1, v2);
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(e1, e2, n);
    sub3(o, v0, w);
    return dot3(n, w) > 0.0;
}

/* global ray id -> (sensor, channel, ray) by the sensor-major layout */
static int decode_ray(const orc_sensor* sensors, uint32_t n_sensors, int64_t g,
                      uint32_t* sn, uint32_t* j, uint32_t* i) {
    if (g < 0) return -1;
    int64_t base = 0;
    for (uint32_t n = 0; n < n_sensors; ++n) {
        int64_t cnt = (int64_t)sensors[n].n_channels * (int64_t)sensors[n].n_rays;
        if (g < base + cnt) {
            int64_t local = g - base;
            *sn = n;
            *j = (uint32_t)(local / sensors[n].n_rays);
            *i = (uint32_t)(local % sensors[n].n_rays);
            return 0;
        }
        base += cnt;
    }
    return -1;
}

typedef struct {
    const orc_sensor* sensors;
    uint32_t n_sensors;
    const float* tris;
    uint32_t n_tris;
    const int64_t* ray_ids;
    int64_t begin, end;
    int cull_backface;
    double tie_rel;
    double* best_t;
    uint32_t* best_id;
    double* second_t;
    uint32_t* n_ties;
    uint32_t* tie_ids;
    uint64_t tests;
    int error;
    const uint8_t* keep;
} cast_job;

static int ray_tri(const orc_sensor* s, const double d[3], const float* tri, int cull, double* t) {
    if (cull && !orc_faces(s->origin, tri)) return 0;
    double tt;
    if (!orc_hit(s->origin, d, tri, &tt)) return 0;
    if (tt < s->d_min || tt > s->d_max) return 0;
    *t = tt;
    return 1;
}

static void* cast_worker(void* arg) {
    cast_job* jb = (cast_job*)arg;
    for (int64_t r = jb->begin; r < jb->end; ++r) {
        uint32_t sn, j, i;
        if (decode_ray(jb->sensors, jb->n_sensors, jb->ray_ids[r], &sn, &j, &i)) {
            jb->error = 1;
            return NULL;
        }
        const orc_sensor* s = &jb->sensors[sn];
        const uint64_t q = (uint64_t)j * s->n_rays + i;
        if (s->mask && !((s->mask[q >> 5] >> (q & 31u)) & 1u)) {
            /* the ray does not fire (App. A.3): a miss */
            jb->best_t[r] = INFINITY;
            jb->best_id[r] = ORC_NO_HIT;
            if (jb->second_t) jb->second_t[r] = INFINITY;
            if (jb->n_ties) jb->n_ties[r] = 0;
            continue;
        }
        double d[3];
        orc_ray_dir(s, j, i, d);
        double best = INFINITY;
        uint32_t bid = ORC_NO_HIT;
        const uint8_t* keep = jb->keep ? jb->keep + (size_t)sn * jb->n_tris : NULL;
        for (uint32_t k = 0; k < jb->n_tris; ++k) {
            double t;
            if (keep && !keep[k]) continue;
            if (ray_tri(s, d, jb->tris + 9 * (size_t)k, jb->cull_backface, &t) && t < best) {
                best = t;
                bid = k;  /* strict '<' over ascending k: ties keep the lower id */
            }
        }
        jb->tests += jb->n_tris;
        jb->best_t[r] = best;
        jb->best_id[r] = bid;
        if (jb->second_t || jb->n_ties) {
            /* second pass: runner-up among other triangles, and the near-tie set */
            double second = INFINITY;
            uint32_t nt = 0;
            double lim = best * (1.0 + jb->tie_rel);
            for (uint32_t k = 0; k < jb->n_tris; ++k) {
                double t;
                if (keep && !keep[k]) continue;
                if (!ray_tri(s, d, jb->tris + 9 * (size_t)k, jb->cull_backface, &t)) continue;
                if (k != bid && t < second) second = t;
                if (bid != ORC_NO_HIT && t <= lim) {
                    if (jb->tie_ids && nt < ORC_MAX_TIES) jb->tie_ids[r * ORC_MAX_TIES + nt] = k;
                    nt++;
                }
            }
            if (jb->second_t) jb->second_t[r] = second;
            if (jb->n_ties) jb->n_ties[r] = nt;
        }
    }
    return NULL;
}

int orc_cast(const orc_sensor* sensors, uint32_t n_sensors, const float* tris, uint32_t n_tris,
             const int64_t* ray_ids, int64_t n_rays, int cull_backface, double tie_rel, int n_threads,
             double* best_t, uint32_t* best_id, double* second_t, uint32_t* n_ties, uint32_t* tie_ids,
             uint64_t* n_tests, const uint8_t* keep) {
    if (!sensors || !n_sensors || (!tris && n_tris) || (!ray_ids && n_rays) || !best_t || !best_id)
        return -1;
    if (n_threads < 1) n_threads = 1;
    if ((int64_t)n_threads > n_rays) n_threads = n_rays > 0 ? (int)n_rays : 1;
    cast_job* jobs = (cast_job*)calloc((size_t)n_threads, sizeof(cast_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        return -1;
    }
    for (int w = 0; w < n_threads; ++w) {
        cast_job* jb = &jobs[w];
        jb->sensors = sensors;
        jb->n_sensors = n_sensors;
        jb->tris = tris;
        jb->n_tris = n_tris;
        jb->ray_ids = ray_ids;
        jb->begin = n_rays * w / n_threads;
        jb->end = n_rays * (w + 1) / n_threads;
        jb->cull_backface = cull_backface;
        jb->tie_rel = tie_rel;
        jb->best_t = best_t;
        jb->best_id = best_id;
        jb->second_t = second_t;
        jb->n_ties = n_ties;
        jb->tie_ids = tie_ids;
        jb->keep = keep;
    }
    for (int w = 1; w < n_threads; ++w) pthread_create(&th[w], NULL, cast_worker, &jobs[w]);
    cast_worker(&jobs[0]);
    for (int w = 1; w < n_threads; ++w) pthread_join(th[w], NULL);
    uint64_t tests = 0;
    int err = 0;
    for (int w = 0; w < n_threads; ++w) {
        tests += jobs[w].tests;
        err |= jobs[w].error;
    }
    if (n_tests) *n_tests = tests;
    free(jobs);
    free(th);
    return err ? -1 : 0;
}

/* Eq. apparent_area (App. A.4.1 Step 1): A_origin = A_T (c-o).n^ / |c-o|^3,
 * compared squared: (A_T (c-o).n^)^2 < eps^2 |c-o|^6 drops the pair. */
void orc_area_keep(const orc_sensor* sensors, uint32_t n_sensors, const float* tris, uint32_t n_tris, double eps,
                   uint8_t* out) {
    for (uint32_t n = 0; n < n_sensors; ++n) {
        const orc_sensor* s = &sensors[n];
        for (uint32_t k = 0; k < n_tris; ++k) {
            double v0[3], v1[3], v2[3], e1[3], e2[3], nrm[3], c[3];
            load_tri(tris + 9 * (size_t)k, v0, v1, v2);
            sub3(v1, v0, e1);
            sub3(v2, v0, e2);
            cross3(e1, e2, nrm);
            double len = sqrt(dot3(nrm, nrm));
            double area = 0.5 * len;
            for (int i = 0; i < 3; ++i) c[i] = (v0[i] + v1[i] + v2[i]) / 3.0 - s->origin[i];
            double cn = len > 0.0 ? dot3(c, nrm) / len : 0.0;
            double lhs = (area * cn) * (area * cn);
            double r2 = dot3(c, c);
            double rhs = eps * eps * r2 * r2 * r2;
            uint8_t v = lhs < rhs ? 0 : 1;
            if (fabs(lhs - rhs) <= 1e-3 * rhs) v = 2;
            out[(size_t)n * n_tris + k] = v;
        }
    }
}

int orc_ray_tri_margin(const orc_sensor* sensors, uint32_t n_sensors, int64_t ray_id,
                       const float* tri, double* t_plane, double* margin) {
    uint32_t sn, j, i;
    if (decode_ray(sensors, n_sensors, ray_id, &sn, &j, &i)) return -1;
    const orc_sensor* s = &sensors[sn];
    double d[3], v0[3], v1[3], v2[3], e1[3], e2[3], n[3], w[3];
    orc_ray_dir(s, j, i, d);
    load_tri(tri, v0, v1, v2);
    sub3(v1, v0, e1);
    sub3(v2, v0, e2);
    cross3(e1, e2, n);
    sub3(v0, s->origin, w);
    double denom = dot3(n, d);
    *t_plane = (denom != 0.0 && dot3(n, n) != 0.0) ? dot3(n, w) / denom : INFINITY;
    /* vertices relative to the origin; the plane through o and edge (a,b) has
     * normal a x b; the interior side is the one holding the third vertex. */
    double p[3][3];
    sub3(v0, s->origin, p[0]);
    sub3(v1, s->origin, p[1]);
    sub3(v2, s->origin, p[2]);
    double m = INFINITY;
    for (int k = 0; k < 3; ++k) {
        const double* a = p[k];
        const double* b = p[(k + 1) % 3];
        const double* c = p[(k + 2) % 3];
        double ab[3];
        cross3(a, b, ab);
        double len = sqrt(dot3(ab, ab));
        if (len == 0.0) {
            m = -INFINITY;  /* edge collinear with o: no side is defined */
            continue;
        }
        double side = dot3(ab, c) >= 0.0 ? 1.0 : -1.0;
        double sv = side * dot3(ab, d) / len;
        if (sv > 1.0) sv = 1.0;
        if (sv < -1.0) sv = -1.0;
        double ang = asin(sv);
        if (ang < m) m = ang;
    }
    *margin = m;
    return 0;
}

typedef struct {
    const orc_sensor* s;
    const float* tris;
    uint32_t begin, end;
    int cull;
    int64_t* out;
    int64_t cap;
    int64_t* counter;   /* shared, guarded by mu */
    pthread_mutex_t* mu;
} hits_job;

static void* hits_worker(void* arg) {
    hits_job* jb = (hits_job*)arg;
    const orc_sensor* s = jb->s;
    int64_t local_cap = 4096, local_n = 0;
    int64_t* local = (int64_t*)malloc((size_t)local_cap * 2 * sizeof(int64_t));
    for (uint32_t k = jb->begin; k < jb->end; ++k) {
        const float* tri = jb->tris + 9 * (size_t)k;
        for (uint32_t j = 0; j < s->n_channels; ++j) {
            for (uint32_t i = 0; i < s->n_rays; ++i) {
                double d[3], t;
                orc_ray_dir(s, j, i, d);
                if (!ray_tri(s, d, tri, jb->cull, &t)) continue;
                if (local_n == local_cap) {
                    local_cap *= 2;
                    local = (int64_t*)realloc(local, (size_t)local_cap * 2 * sizeof(int64_t));
                }
                local[2 * local_n] = k;
                local[2 * local_n + 1] = (int64_t)j * s->n_rays + i;
                local_n++;
            }
        }
    }
    pthread_mutex_lock(jb->mu);
    int64_t at = *jb->counter;
    *jb->counter += local_n;
    pthread_mutex_unlock(jb->mu);
    for (int64_t q = 0; q < local_n; ++q) {
        if (at + q < jb->cap) {
            jb->out[2 * (at + q)] = local[2 * q];
            jb->out[2 * (at + q) + 1] = local[2 * q + 1];
        }
    }
    free(local);
    return NULL;
}

int64_t orc_triangle_hits(const orc_sensor* s, const float* tris, uint32_t n_tris, int cull_backface,
                          int n_threads, int64_t* out, int64_t cap) {
    if (!s || (!tris && n_tris)) return -1;
    if (n_threads < 1) n_threads = 1;
    if ((uint32_t)n_threads > n_tris) n_threads = n_tris ? (int)n_tris : 1;
    hits_job* jobs = (hits_job*)calloc((size_t)n_threads, sizeof(hits_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    pthread_mutex_t mu;
    pthread_mutex_init(&mu, NULL);
    int64_t counter = 0;
    for (int w = 0; w < n_threads; ++w) {
        jobs[w].s = s;
        jobs[w].tris = tris;
        jobs[w].begin = (uint32_t)((uint64_t)n_tris * w / n_threads);
        jobs[w].end = (uint32_t)((uint64_t)n_tris * (w + 1) / n_threads);
        jobs[w].cull = cull_backface;
        jobs[w].out = out;
        jobs[w].cap = out ? cap : 0;
        jobs[w].counter = &counter;
        jobs[w].mu = &mu;
    }
    for (int w = 1; w < n_threads; ++w) pthread_create(&th[w], NULL, hits_worker, &jobs[w]);
    hits_worker(&jobs[0]);
    for (int w = 1; w < n_threads; ++w) pthread_join(th[w], NULL);
    pthread_mutex_destroy(&mu);
    free(jobs);
    free(th);
    return counter;
}

uint64_t orc_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

#define ORC_PI 3.14159265358979323846

void orc_range_noise(uint64_t seed, const int64_t* q, int64_t n, double* z) {
    const double two24 = 16777216.0;
    for (int64_t k = 0; k < n; ++k) {
        uint64_t c = seed + 2ull * (uint64_t)q[k];
        double u1 = ((double)(orc_splitmix64(c) >> 40) + 1.0) / two24;
        double u2 = (double)(orc_splitmix64(c + 1ull) >> 40) / two24;
        z[k] = sqrt(-2.0 * log(u1)) * cos(2.0 * ORC_PI * u2);
    }
}
