/*
 * Search by triplet — plain CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the reconstruction computes.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg load it; the product
 * path never calls it.  It shares no code, header or constant table with
 * the CUDA library.
 *
 * It follows the paper (arXiv 2207.03936) section "Search by triplet":
 *   - "Sort by phi": phi of every hit from a 2-argument arctangent, mapped
 *     onto the unsigned 16-bit range, hits of each module sorted by it;
 *   - "Track seeding and track following": for consecutive module triplets,
 *     seeding (nearest candidates on the neighbouring module, extrapolation
 *     to the third, scatter dx^2+dy^2, best triplet per middle hit under a
 *     threshold), then following of every forming track to the next module,
 *     flagging the hits of extended tracks; a track that misses two
 *     consecutive modules, or reaches the last iteration, becomes a tracklet
 *     (3 hits) or a track (4 or more hits);
 *   - "Tracklet filter": a least-squares fit of each 3-hit tracklet, kept when
 *     the fit is under a threshold and none of its hits is flagged.
 *
 * Readings where the paper is silent (each one also applies to the CUDA path):
 *   R1 atan2: a degree-9 odd polynomial of the Hastings form tabulated in
 *      Abramowitz & Stegun 4.4.49, evaluated on the octant-reduced ratio,
 *      every operation rounded in fp32 (its error against the exact atan on
 *      [0, 1] is at most 1.15e-5 rad, measured in fp64);
 *      phi16 = rint(a * 32768/pi) taken modulo 2^16.
 *   R2 sort key (module, phi16, input index): a stable sort by phi16.
 *   R3 seeding candidates: the unflagged hits of the neighbouring module
 *      nearest to the middle hit in circular phi16 distance; when more than
 *      K exist, all hits whose distance does not exceed the K-th smallest
 *      distance (ties at the boundary are all kept).
 *   R4 third hit: the minimum scatter over ALL unflagged hits of the third
 *      module (a phi window is only an acceleration); best triplet by
 *      (scatter, sorted position of the first hit, of the third hit).
 *   R5 following picks the unflagged hit of the next module with the least
 *      scatter under the threshold (ties: smaller sorted position).
 *   R6 flag conflicts are resolved in one round per step: every extension
 *      claims its new hit and, for a 3-hit track, also its three hits; the
 *      claim key is (float bits of scatter, track key), track key = sorted
 *      position of the seed's middle hit; an extension is kept only when it
 *      holds the minimum key on every hit it claimed.  A 3-hit track with a
 *      flagged hit does not extend.  Seeds do not flag their hits.
 *   R7 tracklet filter: all three hits unflagged and chi2 < C3, then the
 *      same one-round claim among the survivors with key (bits of chi2, key).
 *   R8 fit: straight line x = x0 + tx z, y = y0 + ty z by least squares with
 *      fp32 sums in hit order, chi2 = sum of squared residuals / sigma^2.
 *   R9 output: tracks sorted by their smallest input hit index, hits of a
 *      track in traversal (module) order.
 *   R10 module pairs (the paper works on module pairs and calls them modules,
 *      section "Search by triplet"; its VELO has modules on two sides of the
 *      beam, Fig. 2): when a second plane position module_z2[m] is given,
 *      module m is a pair of one-sided planes, hits with x >= 0 on the plane
 *      at module_z[m] and hits with x < 0 on the plane at module_z2[m].  Every
 *      extrapolation to a module (R4, R5) targets the plane of the hit it is
 *      compared with, so a candidate's scatter is measured at its own plane.
 *      Without module_z2 every module is one plane at module_z[m].
 *
 * Arithmetic: fp32, every operation rounded as written (build with
 * -ffp-contract=off, no fast-math); IEEE division and rounding.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_MAX_MODULES 64

typedef struct {
    int32_t k_doublets;
    float max_scatter_seed;
    float max_scatter_follow;
    float max_chi2_tracklet;
    float hit_sigma;
} sbt_oracle_config;

/* ---------------------------------------------------------------- phi --- */

/* R1: 2-argument arctangent from the odd polynomial atan(t) ~ t*(a1 + a3 t^2
 * + ... + a9 t^8), 0 <= t <= 1 (Hastings form, Abramowitz & Stegun 4.4.49),
 * after reducing (x, y) to the first octant. */
float sbt_oracle_atan2(float y, float x)
{
    const float a1 = 0.9998660f, a3 = -0.3302995f, a5 = 0.1801410f;
    const float a7 = -0.0851330f, a9 = 0.0208351f;
    float ax = fabsf(x);
    float ay = fabsf(y);
    float mx = ax > ay ? ax : ay;
    float mn = ax > ay ? ay : ax;
    if (mx == 0.0f) return 0.0f;
    float t = mn / mx;
    float t2 = t * t;
    float p = a9;
    p = p * t2 + a7;
    p = p * t2 + a5;
    p = p * t2 + a3;
    p = p * t2 + a1;
    p = p * t;
    if (ay > ax) p = 1.5707963267948966f - p;
    if (x < 0.0f) p = 3.14159265358979323846f - p;
    if (y < 0.0f) p = -p;
    return p;
}

/* Section "Sort by phi": [-pi, pi] onto the unsigned 16-bit range, modulo. */
uint16_t sbt_oracle_phi16(float x, float y)
{
    float a = sbt_oracle_atan2(y, x);
    int32_t q = (int32_t)rintf(a * 10430.378350470453f); /* 32768 / pi */
    return (uint16_t)(q & 0xFFFF);
}

void sbt_oracle_phi16_array(const float* x, const float* y, int32_t n, uint16_t* out)
{
    for (int32_t i = 0; i < n; i++) out[i] = sbt_oracle_phi16(x[i], y[i]);
}

/* Circular distance of two phi16 values (modulo arithmetic of the paper). */
int32_t sbt_oracle_phi_distance(uint16_t u, uint16_t v)
{
    int32_t d1 = (int32_t)((uint16_t)(u - v));
    int32_t d2 = (int32_t)((uint16_t)(v - u));
    return d1 < d2 ? d1 : d2;
}

/* ---------------------------------------------------------------- sort --- */

typedef struct {
    int32_t module;
    uint16_t phi;
    int32_t index;
} sort_rec;

static int cmp_sort_rec(const void* pa, const void* pb)
{
    const sort_rec* a = (const sort_rec*)pa;
    const sort_rec* b = (const sort_rec*)pb;
    if (a->module != b->module) return a->module < b->module ? -1 : 1;
    if (a->phi != b->phi) return a->phi < b->phi ? -1 : 1;
    if (a->index != b->index) return a->index < b->index ? -1 : 1;
    return 0;
}

/* R2.  perm[p] = input index of the hit at sorted position p;
 * module_offsets[m] = first sorted position of module m (size M+1). */
int32_t sbt_oracle_sort_event(const float* x, const float* y, const int32_t* module, int32_t n,
                              int32_t M, int32_t* perm, int32_t* module_offsets,
                              uint16_t* phi_sorted)
{
    if (n < 0 || M < 3 || M > OR_MAX_MODULES) return OR_ERR_ARG;
    for (int32_t i = 0; i < n; i++)
        if (module[i] < 0 || module[i] >= M) return OR_ERR_ARG;
    sort_rec* r = (sort_rec*)malloc(sizeof(sort_rec) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; i++) {
        r[i].module = module[i];
        r[i].phi = sbt_oracle_phi16(x[i], y[i]);
        r[i].index = i;
    }
    qsort(r, (size_t)n, sizeof(sort_rec), cmp_sort_rec);
    for (int32_t m = 0; m <= M; m++) module_offsets[m] = 0;
    for (int32_t p = 0; p < n; p++) {
        perm[p] = r[p].index;
        if (phi_sorted) phi_sorted[p] = r[p].phi;
        module_offsets[r[p].module + 1]++;
    }
    for (int32_t m = 0; m < M; m++) module_offsets[m + 1] += module_offsets[m];
    free(r);
    return OR_OK;
}

/* ----------------------------------------------------------------- fit --- */

/* R8: least-squares straight line through n hits given in order.
 * params = (x0, y0, tx, ty) at z = 0; chi2 = sum of squared residuals / sigma^2. */
void sbt_oracle_fit(const float* x, const float* y, const float* z, int32_t n, float sigma,
                    float* params, float* chi2)
{
    float nf = (float)n;
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;
    for (int32_t i = 0; i < n; i++) {
        sx = sx + x[i];
        sy = sy + y[i];
        sz = sz + z[i];
    }
    float xm = sx / nf, ym = sy / nf, zm = sz / nf;
    float szz = 0.0f, szx = 0.0f, szy = 0.0f;
    for (int32_t i = 0; i < n; i++) {
        float dz = z[i] - zm;
        szz = szz + dz * dz;
        szx = szx + dz * (x[i] - xm);
        szy = szy + dz * (y[i] - ym);
    }
    float tx = szx / szz;
    float ty = szy / szz;
    float s = 0.0f;
    for (int32_t i = 0; i < n; i++) {
        float dz = z[i] - zm;
        float rx = (x[i] - xm) - tx * dz;
        float ry = (y[i] - ym) - ty * dz;
        s = s + (rx * rx + ry * ry);
    }
    params[0] = xm - tx * zm;
    params[1] = ym - ty * zm;
    params[2] = tx;
    params[3] = ty;
    *chi2 = s / (sigma * sigma);
}

/* -------------------------------------------------------------- search --- */

typedef struct {
    int32_t hit[OR_MAX_MODULES]; /* sorted positions, traversal order */
    int32_t nhits;
    int32_t skipped;
    int32_t key;
    int32_t alive;
    int32_t cand;   /* candidate hit of this following step, -1 if none */
    float cand_sc;
} or_track;

typedef struct {
    int32_t n, M;
    const float* module_z;
    const float* module_z2; /* second plane of each module pair (x < 0), or NULL */
    const sbt_oracle_config* cfg;
    float *sx, *sy, *sz;
    uint16_t* sphi;
    int32_t* perm;
    int32_t* modoff;
    uint8_t* flag;
    uint64_t* claim;
    or_track* pool;
    int32_t npool;
    int32_t* final_tracks; /* pool indices of finished tracks with >= 4 hits */
    int32_t nfinal;
    int32_t* tracklets;    /* pool indices of finished 3-hit tracks */
    int32_t ntracklets;
    int32_t max_alive;
} or_event;

static uint32_t f32_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* Straight-line extrapolation of the doublet (a, c) to plane z = zt, then the
 * scatter of hit b: dx^2 + dy^2 (section "Track seeding and track following"). */
static void extrapolate(const or_event* E, int32_t a, int32_t c, float zt, float* xp, float* yp)
{
    float dz = E->sz[c] - E->sz[a];
    float tz = (zt - E->sz[c]) / dz;
    *xp = E->sx[c] + (E->sx[c] - E->sx[a]) * tz;
    *yp = E->sy[c] + (E->sy[c] - E->sy[a]) * tz;
}

/* R10: z of the plane that holds hit b (sorted position) of module m. */
static float plane_z(const or_event* E, int32_t m, int32_t b)
{
    if (E->module_z2 && E->sx[b] < 0.0f) return E->module_z2[m];
    return E->module_z[m];
}

static float scatter(const or_event* E, int32_t b, float xp, float yp)
{
    float dx = E->sx[b] - xp;
    float dy = E->sy[b] - yp;
    return dx * dx + dy * dy;
}

static int cmp_int(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Seeding for middle hit c on module s+1 (R3, R4).  Returns 1 and the triplet
 * when a compatible one exists. */
static int seed_for(or_event* E, int32_t s, int32_t c, int32_t* oa, int32_t* ob)
{
    const int32_t o = s, i = s + 2;
    const int32_t o0 = E->modoff[o], o1 = E->modoff[o + 1];
    const int32_t i0 = E->modoff[i], i1 = E->modoff[i + 1];
    int32_t K = E->cfg->k_doublets;
    /* distances of all unflagged hits of module o */
    int32_t nunf = 0;
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(o1 - o0 + 1));
    for (int32_t a = o0; a < o1; a++)
        if (!E->flag[a]) dist[nunf++] = sbt_oracle_phi_distance(E->sphi[a], E->sphi[c]);
    int32_t dmax = 0x7FFFFFFF;
    if (nunf > K) {
        qsort(dist, (size_t)nunf, sizeof(int32_t), cmp_int);
        dmax = dist[K - 1];
    }
    free(dist);
    int found = 0;
    float best_sc = 0.0f;
    int32_t best_a = -1, best_b = -1;
    for (int32_t a = o0; a < o1; a++) {
        if (E->flag[a]) continue;
        if (nunf > K && sbt_oracle_phi_distance(E->sphi[a], E->sphi[c]) > dmax) continue;
        for (int32_t b = i0; b < i1; b++) {
            if (E->flag[b]) continue;
            float xp, yp;
            extrapolate(E, a, c, plane_z(E, i, b), &xp, &yp);
            float sc = scatter(E, b, xp, yp);
            if (!(sc < E->cfg->max_scatter_seed)) continue;
            int better = !found || sc < best_sc ||
                         (sc == best_sc && (a < best_a || (a == best_a && b < best_b)));
            if (better) {
                found = 1;
                best_sc = sc;
                best_a = a;
                best_b = b;
            }
        }
    }
    if (found) {
        *oa = best_a;
        *ob = best_b;
    }
    return found;
}

/*
 * One seeding step s on a single event, every hit unflagged unless flags
 * (indexed by sorted position) says otherwise: the seeds (R3, R4) as sorted
 * positions (a on module s, c on s+1, b on s+2), ordered by c.  Exposed so
 * that the tests can compare it with exhaustive enumeration.
 */
int32_t sbt_oracle_seed_step(const float* x, const float* y, const float* z, const int32_t* module,
                             int32_t n, const float* module_z, const float* module_z2, int32_t M,
                             const sbt_oracle_config* cfg, int32_t s, const uint8_t* flags,
                             int32_t* out_a, int32_t* out_c, int32_t* out_b)
{
    if (n < 0 || M < 3 || M > OR_MAX_MODULES || s < 0 || s + 2 > M - 1) return -1;
    or_event E;
    memset(&E, 0, sizeof(E));
    E.n = n;
    E.M = M;
    E.module_z = module_z;
    E.module_z2 = module_z2;
    E.cfg = cfg;
    size_t nn = (size_t)(n > 0 ? n : 1);
    E.perm = (int32_t*)malloc(sizeof(int32_t) * nn);
    E.modoff = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M + 1));
    E.sphi = (uint16_t*)malloc(sizeof(uint16_t) * nn);
    int32_t cnt = -1;
    if (sbt_oracle_sort_event(x, y, module, n, M, E.perm, E.modoff, E.sphi) == OR_OK) {
        E.sx = (float*)malloc(sizeof(float) * nn);
        E.sy = (float*)malloc(sizeof(float) * nn);
        E.sz = (float*)malloc(sizeof(float) * nn);
        E.flag = (uint8_t*)calloc(nn, 1);
        for (int32_t p = 0; p < n; p++) {
            E.sx[p] = x[E.perm[p]];
            E.sy[p] = y[E.perm[p]];
            E.sz[p] = z[E.perm[p]];
            if (flags) E.flag[p] = flags[p];
        }
        cnt = 0;
        for (int32_t c = E.modoff[s + 1]; c < E.modoff[s + 2]; c++) {
            if (E.flag[c]) continue;
            int32_t a, b;
            if (seed_for(&E, s, c, &a, &b)) {
                out_a[cnt] = a;
                out_c[cnt] = c;
                out_b[cnt] = b;
                cnt++;
            }
        }
        free(E.sx);
        free(E.sy);
        free(E.sz);
        free(E.flag);
    }
    free(E.perm);
    free(E.modoff);
    free(E.sphi);
    return cnt;
}

static void finalize(or_event* E, int32_t ti)
{
    or_track* T = &E->pool[ti];
    T->alive = 0;
    if (T->nhits >= 4)
        E->final_tracks[E->nfinal++] = ti;
    else
        E->tracklets[E->ntracklets++] = ti;
}

static uint64_t claim_key(float score, int32_t key)
{
    return ((uint64_t)f32_bits(score) << 32) | (uint32_t)key;
}

/* Following to module t (R5, R6). */
static void follow(or_event* E, int32_t t)
{
    const int32_t t0 = E->modoff[t], t1 = E->modoff[t + 1];
    /* candidates */
    for (int32_t ti = 0; ti < E->npool; ti++) {
        or_track* T = &E->pool[ti];
        if (!T->alive) continue;
        T->cand = -1;
        if (T->nhits == 3 &&
            (E->flag[T->hit[0]] || E->flag[T->hit[1]] || E->flag[T->hit[2]]))
            continue;
        for (int32_t b = t0; b < t1; b++) {
            if (E->flag[b]) continue;
            float xp, yp;
            extrapolate(E, T->hit[T->nhits - 2], T->hit[T->nhits - 1], plane_z(E, t, b), &xp, &yp);
            float sc = scatter(E, b, xp, yp);
            if (!(sc < E->cfg->max_scatter_follow)) continue;
            if (T->cand < 0 || sc < T->cand_sc) {  /* b ascending: ties keep the smaller */
                T->cand = b;
                T->cand_sc = sc;
            }
        }
    }
    /* claims: minimum key per hit */
    for (int32_t h = 0; h < E->n; h++) E->claim[h] = UINT64_MAX;
    for (int32_t ti = 0; ti < E->npool; ti++) {
        or_track* T = &E->pool[ti];
        if (!T->alive || T->cand < 0) continue;
        uint64_t k = claim_key(T->cand_sc, T->key);
        if (k < E->claim[T->cand]) E->claim[T->cand] = k;
        if (T->nhits == 3)
            for (int j = 0; j < 3; j++)
                if (k < E->claim[T->hit[j]]) E->claim[T->hit[j]] = k;
    }
    /* resolution: decide every extension from the claims alone, then apply */
    int32_t alive = 0;
    for (int32_t ti = 0; ti < E->npool; ti++) {
        or_track* T = &E->pool[ti];
        if (!T->alive) continue;
        int accepted = 0;
        if (T->cand >= 0) {
            uint64_t k = claim_key(T->cand_sc, T->key);
            accepted = E->claim[T->cand] == k;
            if (T->nhits == 3)
                for (int j = 0; j < 3; j++) accepted = accepted && E->claim[T->hit[j]] == k;
        }
        T->cand = accepted ? T->cand : -2; /* -2 marks a miss for the apply pass */
    }
    for (int32_t ti = 0; ti < E->npool; ti++) {
        or_track* T = &E->pool[ti];
        if (!T->alive) continue;
        if (T->cand >= 0) {
            if (T->nhits == 3)
                for (int j = 0; j < 3; j++) E->flag[T->hit[j]] = 1;
            E->flag[T->cand] = 1;
            T->hit[T->nhits++] = T->cand;
            T->skipped = 0;
        } else {
            T->skipped += 1;
        }
        if (T->skipped == 2)
            finalize(E, ti);
        else
            alive++;
    }
    (void)alive;
}

static void count_alive(or_event* E)
{
    int32_t a = 0;
    for (int32_t ti = 0; ti < E->npool; ti++) a += E->pool[ti].alive;
    if (a > E->max_alive) E->max_alive = a;
}

/* Tracklet filter (R7, R8). Returns number of accepted tracklets, their pool
 * indices in acc[]. */
static int32_t tracklet_filter(or_event* E, int32_t* acc)
{
    float* q = (float*)malloc(sizeof(float) * (size_t)(E->ntracklets + 1));
    uint8_t* ok = (uint8_t*)malloc((size_t)(E->ntracklets + 1));
    for (int32_t h = 0; h < E->n; h++) E->claim[h] = UINT64_MAX;
    for (int32_t k = 0; k < E->ntracklets; k++) {
        or_track* T = &E->pool[E->tracklets[k]];
        ok[k] = !E->flag[T->hit[0]] && !E->flag[T->hit[1]] && !E->flag[T->hit[2]];
        if (!ok[k]) continue;
        float hx[3], hy[3], hz[3], prm[4];
        for (int j = 0; j < 3; j++) {
            hx[j] = E->sx[T->hit[j]];
            hy[j] = E->sy[T->hit[j]];
            hz[j] = E->sz[T->hit[j]];
        }
        sbt_oracle_fit(hx, hy, hz, 3, E->cfg->hit_sigma, prm, &q[k]);
        ok[k] = q[k] < E->cfg->max_chi2_tracklet;
        if (!ok[k]) continue;
        uint64_t key = claim_key(q[k], T->key);
        for (int j = 0; j < 3; j++)
            if (key < E->claim[T->hit[j]]) E->claim[T->hit[j]] = key;
    }
    int32_t nacc = 0;
    for (int32_t k = 0; k < E->ntracklets; k++) {
        if (!ok[k]) continue;
        or_track* T = &E->pool[E->tracklets[k]];
        uint64_t key = claim_key(q[k], T->key);
        int win = 1;
        for (int j = 0; j < 3; j++) win = win && E->claim[T->hit[j]] == key;
        if (win) acc[nacc++] = E->tracklets[k];
    }
    free(q);
    free(ok);
    return nacc;
}

typedef struct {
    int32_t minidx;
    int32_t pool;
} out_rec;

static int cmp_out(const void* a, const void* b)
{
    int32_t x = ((const out_rec*)a)->minidx, y = ((const out_rec*)b)->minidx;
    return (x > y) - (x < y);
}

/*
 * Reconstruct one event.  Inputs: n hits (x, y, z, module id in traversal
 * order), module_z[M] plane positions and, for module pairs (R10), the
 * second planes module_z2[M] (NULL: single planes).  Outputs, each with
 * capacity n:
 * track_len[t], track_hits (concatenated input indices of the event),
 * params[4 t], chi2[t], ndof[t].  stats (8 ints, may be NULL): seeds,
 * tracklets, accepted tracklets, tracks (>= 4 hits), max alive forming tracks.
 * Returns the number of tracks or -1 on invalid input.
 */
int32_t sbt_oracle_event(const float* x, const float* y, const float* z, const int32_t* module,
                         int32_t n, const float* module_z, const float* module_z2, int32_t M,
                         const sbt_oracle_config* cfg, int32_t* track_len, int32_t* track_hits,
                         float* params, float* chi2, int32_t* ndof, int32_t* stats)
{
    if (n < 0 || M < 3 || M > OR_MAX_MODULES || cfg->k_doublets < 1) return -1;
    or_event E;
    memset(&E, 0, sizeof(E));
    E.n = n;
    E.M = M;
    E.module_z = module_z;
    E.module_z2 = module_z2;
    E.cfg = cfg;
    size_t nn = (size_t)(n > 0 ? n : 1);
    E.perm = (int32_t*)malloc(sizeof(int32_t) * nn);
    E.modoff = (int32_t*)malloc(sizeof(int32_t) * (size_t)(M + 1));
    E.sphi = (uint16_t*)malloc(sizeof(uint16_t) * nn);
    if (sbt_oracle_sort_event(x, y, module, n, M, E.perm, E.modoff, E.sphi) != OR_OK) {
        free(E.perm);
        free(E.modoff);
        free(E.sphi);
        return -1;
    }
    E.sx = (float*)malloc(sizeof(float) * nn);
    E.sy = (float*)malloc(sizeof(float) * nn);
    E.sz = (float*)malloc(sizeof(float) * nn);
    for (int32_t p = 0; p < n; p++) {
        E.sx[p] = x[E.perm[p]];
        E.sy[p] = y[E.perm[p]];
        E.sz[p] = z[E.perm[p]];
    }
    E.flag = (uint8_t*)calloc(nn, 1); /* the flagged-hits container starts empty */
    E.claim = (uint64_t*)malloc(sizeof(uint64_t) * nn);
    E.pool = (or_track*)malloc(sizeof(or_track) * nn); /* <= one seed per middle hit */
    E.final_tracks = (int32_t*)malloc(sizeof(int32_t) * nn);
    E.tracklets = (int32_t*)malloc(sizeof(int32_t) * nn);
    int32_t nseeds = 0;

    /* iterative seeding and following over module triplets (s, s+1, s+2) */
    for (int32_t s = 0; s + 2 <= M - 1; s++) {
        for (int32_t c = E.modoff[s + 1]; c < E.modoff[s + 2]; c++) {
            if (E.flag[c]) continue;
            int32_t a, b;
            if (seed_for(&E, s, c, &a, &b)) {
                or_track* T = &E.pool[E.npool++];
                T->hit[0] = a;
                T->hit[1] = c;
                T->hit[2] = b;
                T->nhits = 3;
                T->skipped = 0;
                T->key = c;
                T->alive = 1;
                T->cand = -1;
                nseeds++;
            }
        }
        count_alive(&E);
        if (s + 3 <= M - 1) {
            follow(&E, s + 3);
        } else {
            for (int32_t ti = 0; ti < E.npool; ti++)
                if (E.pool[ti].alive) finalize(&E, ti);
        }
    }

    int32_t* acc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E.ntracklets + 1));
    int32_t nacc = tracklet_filter(&E, acc);

    /* output (R9) */
    int32_t nout = E.nfinal + nacc;
    out_rec* outs = (out_rec*)malloc(sizeof(out_rec) * (size_t)(nout + 1));
    for (int32_t k = 0; k < nout; k++) {
        int32_t pi = k < E.nfinal ? E.final_tracks[k] : acc[k - E.nfinal];
        or_track* T = &E.pool[pi];
        int32_t mn = 0x7FFFFFFF;
        for (int32_t j = 0; j < T->nhits; j++)
            if (E.perm[T->hit[j]] < mn) mn = E.perm[T->hit[j]];
        outs[k].minidx = mn;
        outs[k].pool = pi;
    }
    qsort(outs, (size_t)nout, sizeof(out_rec), cmp_out);
    int32_t w = 0;
    for (int32_t k = 0; k < nout; k++) {
        or_track* T = &E.pool[outs[k].pool];
        float hx[OR_MAX_MODULES], hy[OR_MAX_MODULES], hz[OR_MAX_MODULES];
        for (int32_t j = 0; j < T->nhits; j++) {
            int32_t in = E.perm[T->hit[j]];
            track_hits[w + j] = in;
            hx[j] = x[in];
            hy[j] = y[in];
            hz[j] = z[in];
        }
        w += T->nhits;
        track_len[k] = T->nhits;
        sbt_oracle_fit(hx, hy, hz, T->nhits, cfg->hit_sigma, &params[4 * k], &chi2[k]);
        ndof[k] = 2 * T->nhits - 4;
    }
    if (stats) {
        stats[0] = nseeds;
        stats[1] = E.ntracklets;
        stats[2] = nacc;
        stats[3] = E.nfinal;
        stats[4] = E.max_alive;
        stats[5] = w;
        stats[6] = 0;
        stats[7] = 0;
    }
    free(outs);
    free(acc);
    free(E.perm);
    free(E.modoff);
    free(E.sphi);
    free(E.sx);
    free(E.sy);
    free(E.sz);
    free(E.flag);
    free(E.claim);
    free(E.pool);
    free(E.final_tracks);
    free(E.tracklets);
    return nout;
}

/* ------------------------------------------------------- batch driver --- */

typedef struct {
    const float *x, *y, *z;
    const int32_t* module;
    const int32_t* event_offsets;
    int32_t n_events;
    const float* module_z;
    const float* module_z2;
    int32_t M;
    const sbt_oracle_config* cfg;
    int32_t* ev_ntracks;
    int32_t* ev_nhits;
    int32_t* ev_status;
    int32_t* slot_len;
    int32_t* slot_hits;
    float* slot_params;
    float* slot_chi2;
    int32_t* slot_ndof;
    int32_t* ev_stats;
    int32_t next;
    pthread_mutex_t lock;
} batch_job;

static void* batch_worker(void* arg)
{
    batch_job* J = (batch_job*)arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int32_t e = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (e >= J->n_events) break;
        int32_t off = J->event_offsets[e];
        int32_t n = J->event_offsets[e + 1] - off;
        int32_t tslot = off / 3;
        int32_t nt = sbt_oracle_event(J->x + off, J->y + off, J->z + off, J->module + off, n,
                                      J->module_z, J->module_z2, J->M, J->cfg, J->slot_len + tslot,
                                      J->slot_hits + off, J->slot_params + 4 * (int64_t)tslot,
                                      J->slot_chi2 + tslot, J->slot_ndof + tslot,
                                      J->ev_stats ? J->ev_stats + 8 * (int64_t)e : NULL);
        if (nt < 0) {
            J->ev_status[e] = OR_ERR_ARG;
            J->ev_ntracks[e] = 0;
            J->ev_nhits[e] = 0;
            continue;
        }
        int32_t h = 0;
        for (int32_t k = 0; k < nt; k++) h += J->slot_len[tslot + k];
        /* local -> batch-global hit indices */
        for (int32_t k = 0; k < h; k++) J->slot_hits[off + k] += off;
        J->ev_status[e] = OR_OK;
        J->ev_ntracks[e] = nt;
        J->ev_nhits[e] = h;
    }
    return NULL;
}

/*
 * Reconstruct a batch on n_threads host threads (one event per thread at a
 * time).  Per-event outputs are written into slots: the tracks of event e
 * start at track slot event_offsets[e] / 3 and its hit indices (batch-global)
 * at event_offsets[e]; slot arrays need capacity n_hits (hits) and
 * n_hits / 3 + n_events (tracks).
 */
int32_t sbt_oracle_batch(const float* x, const float* y, const float* z, const int32_t* module,
                         const int32_t* event_offsets, int32_t n_events, const float* module_z,
                         const float* module_z2, int32_t M, const sbt_oracle_config* cfg,
                         int32_t n_threads,
                         int32_t* ev_ntracks, int32_t* ev_nhits, int32_t* ev_status,
                         int32_t* slot_len, int32_t* slot_hits, float* slot_params,
                         float* slot_chi2, int32_t* slot_ndof, int32_t* ev_stats)
{
    batch_job J;
    memset(&J, 0, sizeof(J));
    J.x = x; J.y = y; J.z = z; J.module = module; J.event_offsets = event_offsets;
    J.n_events = n_events; J.module_z = module_z; J.module_z2 = module_z2; J.M = M; J.cfg = cfg;
    J.ev_ntracks = ev_ntracks; J.ev_nhits = ev_nhits; J.ev_status = ev_status;
    J.slot_len = slot_len; J.slot_hits = slot_hits; J.slot_params = slot_params;
    J.slot_chi2 = slot_chi2; J.slot_ndof = slot_ndof; J.ev_stats = ev_stats;
    pthread_mutex_init(&J.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 512) n_threads = 512;
    pthread_t th[512];
    for (int32_t i = 0; i < n_threads; i++) pthread_create(&th[i], NULL, batch_worker, &J);
    for (int32_t i = 0; i < n_threads; i++) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&J.lock);
    return n_threads;
}

/* ----------------------------------------------------- alignment chi2 --- */

/*
 * Summed chi2 of fixed tracks after per-module alignment, in fp64 (the
 * differentiation workload; the paper's fit of the tracklet filter applied
 * to every track).  For a hit h on module m with plane centre c = (0, 0,
 * module_z[m]) and parameters (dx, dy, dz, a, b, g) = align[6 m .. 6 m + 5]:
 *     h' = Rz(g) Ry(b) Rx(a) (h - c) + c + (dx, dy, dz).
 * Each track is refitted by least squares on the aligned hits; the return
 * value is sum over tracks of sum of squared residuals / sigma^2.  When grad
 * is not NULL it receives d(chi2 sum)/d(align) [M * 6], using that at the
 * least-squares optimum the derivative with respect to each hit is the
 * partial derivative at fixed line parameters.
 *
 * A track takes part when it has a straight-line fit: at least two hits,
 * hits on at least two modules, every hit index in [0, n_hits), every module
 * id in [0, M), and its hit range inside [0, hit_offsets[n_tracks]).  Other
 * tracks contribute nothing; *skipped (may be NULL) receives their number.
 * A track may have any number of hits, several on one module included.
 */
double sbt_oracle_align_chi2(const float* x, const float* y, const float* z, const int32_t* module,
                             int32_t n_hits, const int32_t* hit_offsets, const int32_t* track_hits,
                             int32_t n_tracks, const float* module_z, int32_t M,
                             const double* align, double sigma, double* grad, int32_t* skipped)
{
    double total = 0.0;
    int32_t nskip = 0;
    if (grad)
        for (int32_t k = 0; k < 6 * M; k++) grad[k] = 0.0;
    double s2 = sigma * sigma;
    const int64_t end = n_tracks > 0 ? hit_offsets[n_tracks] : 0;
    int32_t cap = 0;
    double *px = NULL, *py = NULL, *pz = NULL, *lx = NULL, *ly = NULL, *lz = NULL;
    int32_t* mod = NULL;
    for (int32_t t = 0; t < n_tracks; t++) {
        int32_t h0 = hit_offsets[t], n = hit_offsets[t + 1] - hit_offsets[t];
        int ok = n >= 2 && h0 >= 0 && (int64_t)h0 + n <= end;
        for (int32_t j = 0; ok && j < n; j++) {
            int32_t h = track_hits[h0 + j];
            ok = h >= 0 && h < n_hits && module[h] >= 0 && module[h] < M;
        }
        if (ok) {
            int two = 0;
            for (int32_t j = 1; j < n; j++) two = two || module[track_hits[h0 + j]] != module[track_hits[h0]];
            ok = two;
        }
        if (!ok) {
            nskip++;
            continue;
        }
        if (n > cap) {
            cap = n;
            px = (double*)realloc(px, sizeof(double) * (size_t)cap);
            py = (double*)realloc(py, sizeof(double) * (size_t)cap);
            pz = (double*)realloc(pz, sizeof(double) * (size_t)cap);
            lx = (double*)realloc(lx, sizeof(double) * (size_t)cap);
            ly = (double*)realloc(ly, sizeof(double) * (size_t)cap);
            lz = (double*)realloc(lz, sizeof(double) * (size_t)cap);
            mod = (int32_t*)realloc(mod, sizeof(int32_t) * (size_t)cap);
        }
        for (int32_t j = 0; j < n; j++) {
            int32_t h = track_hits[h0 + j];
            int32_t m = module[h];
            const double* th = align + 6 * m;
            double ca = cos(th[3]), sa = sin(th[3]);
            double cb = cos(th[4]), sb = sin(th[4]);
            double cg = cos(th[5]), sg = sin(th[5]);
            double vx = (double)x[h], vy = (double)y[h], vz = (double)z[h] - (double)module_z[m];
            lx[j] = vx; ly[j] = vy; lz[j] = vz;
            /* Rx */
            double ax = vx, ay = ca * vy - sa * vz, az = sa * vy + ca * vz;
            /* Ry */
            double bx = cb * ax + sb * az, by = ay, bz = -sb * ax + cb * az;
            /* Rz */
            double gx = cg * bx - sg * by, gy = sg * bx + cg * by, gz = bz;
            px[j] = gx + th[0];
            py[j] = gy + th[1];
            pz[j] = gz + (double)module_z[m] + th[2];
            mod[j] = m;
        }
        double sx = 0, sy = 0, sz = 0;
        for (int32_t j = 0; j < n; j++) { sx += px[j]; sy += py[j]; sz += pz[j]; }
        double xm = sx / n, ym = sy / n, zm = sz / n;
        double szz = 0, szx = 0, szy = 0;
        for (int32_t j = 0; j < n; j++) {
            double dz = pz[j] - zm;
            szz += dz * dz;
            szx += dz * (px[j] - xm);
            szy += dz * (py[j] - ym);
        }
        double tx = szx / szz, ty = szy / szz;
        for (int32_t j = 0; j < n; j++) {
            double dz = pz[j] - zm;
            double rx = (px[j] - xm) - tx * dz;
            double ry = (py[j] - ym) - ty * dz;
            total += (rx * rx + ry * ry) / s2;
            if (!grad) continue;
            double gx = 2.0 * rx / s2, gy = 2.0 * ry / s2, gz = -(2.0 * rx * tx + 2.0 * ry * ty) / s2;
            int32_t m = mod[j];
            const double* th = align + 6 * m;
            double ca = cos(th[3]), sa = sin(th[3]);
            double cb = cos(th[4]), sb = sin(th[4]);
            double cg = cos(th[5]), sg = sin(th[5]);
            double vx = lx[j], vy = ly[j], vz = lz[j];
            double* G = grad + 6 * m;
            G[0] += gx;
            G[1] += gy;
            G[2] += gz;
            /* d/da: Rz Ry dRx v */
            {
                double ax = 0.0, ay = -sa * vy - ca * vz, az = ca * vy - sa * vz;
                double bx = cb * ax + sb * az, by = ay, bz = -sb * ax + cb * az;
                double ux = cg * bx - sg * by, uy = sg * bx + cg * by, uz = bz;
                G[3] += gx * ux + gy * uy + gz * uz;
            }
            /* d/db: Rz dRy Rx v */
            {
                double ax = vx, ay = ca * vy - sa * vz, az = sa * vy + ca * vz;
                double bx = -sb * ax + cb * az, by = 0.0, bz = -cb * ax - sb * az;
                double ux = cg * bx - sg * by, uy = sg * bx + cg * by, uz = bz;
                G[4] += gx * ux + gy * uy + gz * uz;
            }
            /* d/dg: dRz Ry Rx v */
            {
                double ax = vx, ay = ca * vy - sa * vz, az = sa * vy + ca * vz;
                double bx = cb * ax + sb * az, by = ay;
                double ux = -sg * bx - cg * by, uy = cg * bx - sg * by;
                G[5] += gx * ux + gy * uy;
            }
        }
    }
    free(px);
    free(py);
    free(pz);
    free(lx);
    free(ly);
    free(lz);
    free(mod);
    if (skipped) *skipped = nskip;
    return total;
}
