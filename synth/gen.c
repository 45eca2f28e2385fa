/*
 * gen.c -- seeded synthetic segmentation volumes that stand in for the
 * paper's data sets (Cells, Fiber, Cortex are not available).  This module
 * holds no codec arithmetic: it only makes uint32 label volumes, x fastest,
 * that both the CPU oracle and the CUDA library consume.
 *
 * Randomness: splitmix64 (Steele, Lea, Flood 2014) as a stream generator and
 * its output mix as a hash.  Geometry of the Voronoi generators is exact
 * integer arithmetic in 1/256-voxel fixed point, so results do not depend on
 * floating point or thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

#define GOLDEN 0x9E3779B97F4A7C15ull

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t sm_next(uint64_t *s) {
    *s += GOLDEN;
    return mix64(*s);
}

static uint64_t hash2(uint64_t a, uint64_t b) { return mix64(mix64(a + GOLDEN) ^ (b * GOLDEN + 0x632BE59BD9B4E019ull)); }

/* label of object id under seed: a hashed uint32, never 0 (0 is background) */
uint32_t synth_label(uint64_t seed, uint64_t id) {
    uint32_t v = (uint32_t)hash2(seed ^ 0x5EED1AB1ull, id);
    return v ? v : 1u;
}

/* ------------------------------------------------------------------ */
/* threading helper: split z slices over threads                       */
/* ------------------------------------------------------------------ */

typedef void (*slab_fn)(void *ctx, uint64_t z0, uint64_t z1);
typedef struct {
    slab_fn fn;
    void *ctx;
    uint64_t Z, next;
    pthread_mutex_t mu;
} slab_job;

static void *slab_worker(void *arg) {
    slab_job *J = (slab_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        uint64_t z = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (z >= J->Z) break;
        J->fn(J->ctx, z, z + 1);
    }
    return NULL;
}

static void run_slabs(slab_fn fn, void *ctx, uint64_t Z, int n_threads) {
    slab_job J = {fn, ctx, Z, 0};
    pthread_mutex_init(&J.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    for (int i = 0; i < n_threads; i++) pthread_create(&th[i], NULL, slab_worker, &J);
    for (int i = 0; i < n_threads; i++) pthread_join(th[i], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
}

/* ------------------------------------------------------------------ */
/* Voronoi partition, optionally warped by value noise, with           */
/* background cells                                                    */
/* ------------------------------------------------------------------ */

#define FP 256 /* fixed point: 1/256 voxel */
#define CELL 16 /* site grid cell, voxels */

typedef struct {
    uint32_t *vol;
    uint64_t X, Y, Z;
    uint64_t seed;
    uint32_t n_sites;
    int64_t *sx, *sy, *sz; /* site coordinates, fixed point */
    uint32_t *label;       /* label per site (0 = background) */
    /* site grid: CSR over cells */
    int64_t gx, gy, gz;
    uint32_t *cell_start, *cell_sites;
    /* warp noise */
    int warp_amp; /* voxels; 0 = none */
    int periods[3];
    int16_t *lat[3][3]; /* [octave][axis] lattice values in [-256, 256] */
    int64_t lat_n[3][3]; /* lattice side per octave (same for all axes) */
} vor_ctx;

static int16_t lattice_value(uint64_t seed, int octave, int axis, int64_t i, int64_t j, int64_t k) {
    uint64_t key = ((uint64_t)(octave * 3 + axis) << 60) ^ ((uint64_t)i << 40) ^ ((uint64_t)j << 20) ^ (uint64_t)k;
    return (int16_t)((int64_t)(hash2(seed ^ 0xC0FFEEull, key) % 513u) - 256);
}

/* displacement along axis a at integer voxel (x,y,z), in 1/256 voxel */
static int64_t warp_disp(const vor_ctx *V, int a, int64_t x, int64_t y, int64_t z) {
    static const int64_t weight[3] = {4, 2, 1};
    int64_t acc = 0;
    for (int o = 0; o < 3; o++) {
        int64_t P = V->periods[o], n = V->lat_n[o][a];
        const int16_t *L = V->lat[o][a];
        int64_t i0 = x / P, j0 = y / P, k0 = z / P;
        int64_t fx = (x % P) * FP / P, fy = (y % P) * FP / P, fz = (z % P) * FP / P;
        int64_t c[2][2];
        for (int dk = 0; dk < 2; dk++)
            for (int dj = 0; dj < 2; dj++) {
                int64_t base = ((k0 + dk) * n + (j0 + dj)) * n + i0;
                c[dk][dj] = (int64_t)L[base] * (FP - fx) + (int64_t)L[base + 1] * fx;
            }
        int64_t e0 = c[0][0] * (FP - fy) + c[0][1] * fy;
        int64_t e1 = c[1][0] * (FP - fy) + c[1][1] * fy;
        int64_t v = e0 * (FP - fz) + e1 * fz; /* units 256^3 * [-256,256] */
        acc += weight[o] * (v / (FP * FP));   /* -> [-256*256, 256*256] */
    }
    /* normalise weights (4+2+1) and scale to the amplitude: [-256,256] * amp voxels */
    return (acc / 7) * V->warp_amp / FP;
}

static void vor_slab(void *ctx, uint64_t z0, uint64_t z1) {
    const vor_ctx *V = (const vor_ctx *)ctx;
    for (uint64_t z = z0; z < z1; z++)
        for (uint64_t y = 0; y < V->Y; y++)
            for (uint64_t x = 0; x < V->X; x++) {
                int64_t px = (int64_t)x * FP + FP / 2, py = (int64_t)y * FP + FP / 2, pz = (int64_t)z * FP + FP / 2;
                if (V->warp_amp) {
                    px += warp_disp(V, 0, x, y, z);
                    py += warp_disp(V, 1, x, y, z);
                    pz += warp_disp(V, 2, x, y, z);
                }
                /* cell of p, possibly outside the grid (floor division) */
                int64_t S = (int64_t)CELL * FP;
                int64_t cx = (px >= 0) ? px / S : -((-px + S - 1) / S);
                int64_t cy = (py >= 0) ? py / S : -((-py + S - 1) / S);
                int64_t cz = (pz >= 0) ? pz / S : -((-pz + S - 1) / S);
                int64_t best = INT64_MAX;
                uint32_t best_id = 0;
                for (int64_t r = 0;; r++) {
                    for (int64_t kz = cz - r; kz <= cz + r; kz++)
                        for (int64_t ky = cy - r; ky <= cy + r; ky++)
                            for (int64_t kx = cx - r; kx <= cx + r; kx++) {
                                int64_t dx = kx - cx, dy = ky - cy, dz = kz - cz;
                                int64_t cheb = dx < 0 ? -dx : dx;
                                if ((dy < 0 ? -dy : dy) > cheb) cheb = dy < 0 ? -dy : dy;
                                if ((dz < 0 ? -dz : dz) > cheb) cheb = dz < 0 ? -dz : dz;
                                if (cheb != r) continue; /* only the shell */
                                if (kx < 0 || ky < 0 || kz < 0 || kx >= V->gx || ky >= V->gy || kz >= V->gz) continue;
                                int64_t ci = (kz * V->gy + ky) * V->gx + kx;
                                for (uint32_t s = V->cell_start[ci]; s < V->cell_start[ci + 1]; s++) {
                                    uint32_t id = V->cell_sites[s];
                                    int64_t ex = V->sx[id] - px, ey = V->sy[id] - py, ez = V->sz[id] - pz;
                                    int64_t d2 = ex * ex + ey * ey + ez * ez;
                                    if (d2 < best || (d2 == best && id < best_id)) { best = d2; best_id = id; }
                                }
                            }
                    /* every site in shell r+1 or beyond is at least r*S away */
                    if (best != INT64_MAX && best <= (r * S) * (r * S)) break;
                    if (r > V->gx + V->gy + V->gz + 4) break;
                }
                V->vol[x + V->X * (y + V->Y * z)] = V->label[best_id];
            }
}

/*
 * Voronoi partition of n_sites sites uniform in the volume (fixed point);
 * nearest site by exact squared distance from voxel centres, ties to the
 * lower site id.  warp_amp > 0 displaces each voxel centre by 3-octave value
 * noise (periods 32/16/8 voxels, weights 4:2:1, amplitude warp_amp voxels per
 * axis).  A site's cell is background (label 0) with probability
 * bg_permille/1000; other cells get synth_label(seed, site).
 */
int synth_voronoi(uint32_t *vol, uint64_t X, uint64_t Y, uint64_t Z, uint32_t n_sites, uint64_t seed,
                  int warp_amp, uint32_t bg_permille, int n_threads) {
    if (!n_sites || !X || !Y || !Z) return 1;
    vor_ctx V;
    memset(&V, 0, sizeof V);
    V.vol = vol; V.X = X; V.Y = Y; V.Z = Z; V.seed = seed; V.n_sites = n_sites; V.warp_amp = warp_amp;
    V.sx = (int64_t *)malloc(8 * n_sites);
    V.sy = (int64_t *)malloc(8 * n_sites);
    V.sz = (int64_t *)malloc(8 * n_sites);
    V.label = (uint32_t *)malloc(4 * n_sites);
    uint64_t st = seed;
    for (uint32_t i = 0; i < n_sites; i++) {
        V.sx[i] = (int64_t)(sm_next(&st) % (X * FP));
        V.sy[i] = (int64_t)(sm_next(&st) % (Y * FP));
        V.sz[i] = (int64_t)(sm_next(&st) % (Z * FP));
        int bg = (hash2(seed ^ 0xBA5E0ull, i) % 1000u) < bg_permille;
        V.label[i] = bg ? 0u : synth_label(seed, i);
    }
    V.gx = (int64_t)((X + CELL - 1) / CELL);
    V.gy = (int64_t)((Y + CELL - 1) / CELL);
    V.gz = (int64_t)((Z + CELL - 1) / CELL);
    int64_t ncell = V.gx * V.gy * V.gz;
    V.cell_start = (uint32_t *)calloc(ncell + 1, 4);
    V.cell_sites = (uint32_t *)malloc(4 * n_sites);
    int64_t *cell_of = (int64_t *)malloc(8 * n_sites);
    for (uint32_t i = 0; i < n_sites; i++) {
        int64_t ci = ((V.sz[i] / (CELL * FP)) * V.gy + V.sy[i] / (CELL * FP)) * V.gx + V.sx[i] / (CELL * FP);
        cell_of[i] = ci;
        V.cell_start[ci + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) V.cell_start[c + 1] += V.cell_start[c];
    uint32_t *fill = (uint32_t *)calloc(ncell, 4);
    for (uint32_t i = 0; i < n_sites; i++) V.cell_sites[V.cell_start[cell_of[i]] + fill[cell_of[i]]++] = i;
    free(fill);
    free(cell_of);
    if (warp_amp) {
        V.periods[0] = 32; V.periods[1] = 16; V.periods[2] = 8;
        uint64_t side = X > Y ? X : Y;
        side = side > Z ? side : Z;
        for (int o = 0; o < 3; o++)
            for (int a = 0; a < 3; a++) {
                int64_t n = (int64_t)(side / V.periods[o]) + 2;
                V.lat_n[o][a] = n;
                V.lat[o][a] = (int16_t *)malloc(2 * n * n * n);
                for (int64_t k = 0; k < n; k++)
                    for (int64_t j = 0; j < n; j++)
                        for (int64_t i = 0; i < n; i++)
                            V.lat[o][a][(k * n + j) * n + i] = lattice_value(seed, o, a, i, j, k);
            }
    }
    run_slabs(vor_slab, &V, Z, n_threads);
    free(V.sx); free(V.sy); free(V.sz); free(V.label); free(V.cell_start); free(V.cell_sites);
    for (int o = 0; o < 3; o++)
        for (int a = 0; a < 3; a++) free(V.lat[o][a]);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Elongated ellipsoid "cells" packed by rejection                     */
/* ------------------------------------------------------------------ */

static double u01(uint64_t *s) { return (double)(sm_next(s) >> 11) * (1.0 / 9007199254740992.0); }

typedef struct {
    double c[3];
    double R[3][3]; /* rows: principal axes */
    double inv2[3]; /* 1 / semi-axis^2 */
    int64_t lo[3], hi[3];
} ellipsoid;

static int inside(const ellipsoid *e, int64_t x, int64_t y, int64_t z) {
    double d[3] = {x + 0.5 - e->c[0], y + 0.5 - e->c[1], z + 0.5 - e->c[2]};
    double q = 0;
    for (int k = 0; k < 3; k++) {
        double u = e->R[k][0] * d[0] + e->R[k][1] * d[1] + e->R[k][2] * d[2];
        q += u * u * e->inv2[k];
    }
    return q <= 1.0;
}

/*
 * Pack up to n_target ellipsoids into an empty (label 0) volume by
 * rejection against a voxel occupancy bitmap, sequentially (deterministic).
 * Long axis length U[len_lo, len_hi] voxels, the two short axes U[short_lo,
 * long/2]; orientation a uniform random unit quaternion; centres uniform.
 * Returns the number placed; vol must be zeroed by the caller.
 */
uint64_t synth_ellipsoids(uint32_t *vol, uint64_t X, uint64_t Y, uint64_t Z, uint64_t n_target, uint64_t seed,
                          double len_lo, double len_hi, double short_lo, uint64_t max_attempts) {
    uint64_t nvox = X * Y * Z;
    uint8_t *occ = (uint8_t *)calloc((nvox + 7) / 8, 1);
    uint64_t st = seed, placed = 0;
    for (uint64_t att = 0; att < max_attempts && placed < n_target; att++) {
        ellipsoid e;
        double len = len_lo + (len_hi - len_lo) * u01(&st);
        double s1 = short_lo + (len / 2 - short_lo) * u01(&st);
        double s2 = short_lo + (len / 2 - short_lo) * u01(&st);
        double a[3] = {len / 2, s1 / 2, s2 / 2};
        /* uniform quaternion (Shoemake) */
        double u1 = u01(&st), u2 = u01(&st), u3 = u01(&st);
        double qw = sqrt(1 - u1) * sin(2 * M_PI * u2), qx = sqrt(1 - u1) * cos(2 * M_PI * u2);
        double qy = sqrt(u1) * sin(2 * M_PI * u3), qz = sqrt(u1) * cos(2 * M_PI * u3);
        double R[3][3] = {{1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)},
                          {2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)},
                          {2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)}};
        e.c[0] = u01(&st) * X; e.c[1] = u01(&st) * Y; e.c[2] = u01(&st) * Z;
        for (int k = 0; k < 3; k++) {
            for (int j = 0; j < 3; j++) e.R[k][j] = R[j][k];
            e.inv2[k] = 1.0 / (a[k] * a[k]);
        }
        int ok = 1;
        for (int j = 0; j < 3; j++) {
            /* half extent along world axis j */
            double h = 0;
            for (int k = 0; k < 3; k++) h += (a[k] * e.R[k][j]) * (a[k] * e.R[k][j]);
            h = sqrt(h);
            double dim = j == 0 ? (double)X : j == 1 ? (double)Y : (double)Z;
            e.lo[j] = (int64_t)floor(e.c[j] - h - 0.5);
            e.hi[j] = (int64_t)ceil(e.c[j] + h + 0.5);
            if (e.lo[j] < 0 || e.hi[j] > (int64_t)dim) ok = 0; /* keep cells inside the volume */
        }
        if (!ok) continue;
        for (int64_t z = e.lo[2]; z < e.hi[2] && ok; z++)
            for (int64_t y = e.lo[1]; y < e.hi[1] && ok; y++)
                for (int64_t x = e.lo[0]; x < e.hi[0]; x++) {
                    uint64_t i = (uint64_t)x + X * ((uint64_t)y + Y * (uint64_t)z);
                    if ((occ[i >> 3] >> (i & 7)) & 1) {
                        if (inside(&e, x, y, z)) { ok = 0; break; }
                    }
                }
        if (!ok) continue;
        uint32_t lab = synth_label(seed, placed);
        for (int64_t z = e.lo[2]; z < e.hi[2]; z++)
            for (int64_t y = e.lo[1]; y < e.hi[1]; y++)
                for (int64_t x = e.lo[0]; x < e.hi[0]; x++)
                    if (inside(&e, x, y, z)) {
                        uint64_t i = (uint64_t)x + X * ((uint64_t)y + Y * (uint64_t)z);
                        occ[i >> 3] |= (uint8_t)(1u << (i & 7));
                        vol[i] = lab;
                    }
        placed++;
    }
    free(occ);
    return placed;
}

/* ------------------------------------------------------------------ */
/* Worley F1 cells on a jittered grid                                  */
/* ------------------------------------------------------------------ */

/*
 * Feature point of grid cell (i,j,k), cell side C voxels: the cell origin
 * plus a hashed jitter in [0, C) per axis, in 1/256 voxel.  Shared formula
 * with gen_gpu.cu (same integers on both sides).
 */
static void worley_feature(uint64_t seed, int64_t i, int64_t j, int64_t k, int64_t C, int64_t f[3]) {
    uint64_t key = ((uint64_t)(i + 1) << 42) ^ ((uint64_t)(j + 1) << 21) ^ (uint64_t)(k + 1);
    uint64_t h = hash2(seed ^ 0x3A0E1Eull, key);
    f[0] = i * C * FP + (int64_t)((h & 0xFFFFFull) % (uint64_t)(C * FP));
    f[1] = j * C * FP + (int64_t)(((h >> 20) & 0xFFFFFull) % (uint64_t)(C * FP));
    f[2] = k * C * FP + (int64_t)(((h >> 40) & 0xFFFFFull) % (uint64_t)(C * FP));
}

typedef struct {
    uint32_t *vol;
    uint64_t X, Y, Z, seed;
    int64_t C;
} worley_ctx;

static void worley_slab(void *ctx, uint64_t z0, uint64_t z1) {
    const worley_ctx *W = (const worley_ctx *)ctx;
    for (uint64_t z = z0; z < z1; z++)
        for (uint64_t y = 0; y < W->Y; y++)
            for (uint64_t x = 0; x < W->X; x++) {
                int64_t p[3] = {(int64_t)x * FP + FP / 2, (int64_t)y * FP + FP / 2, (int64_t)z * FP + FP / 2};
                int64_t ci = (int64_t)x / W->C, cj = (int64_t)y / W->C, ck = (int64_t)z / W->C;
                int64_t best = INT64_MAX, bi = 0, bj = 0, bk = 0;
                /* the 27 neighbouring cells; ties go to the lexicographically smallest (i, j, k) */
                for (int64_t i = ci - 1; i <= ci + 1; i++)
                    for (int64_t j = cj - 1; j <= cj + 1; j++)
                        for (int64_t k = ck - 1; k <= ck + 1; k++) {
                            int64_t f[3];
                            worley_feature(W->seed, i, j, k, W->C, f);
                            int64_t d0 = f[0] - p[0], d1 = f[1] - p[1], d2 = f[2] - p[2];
                            int64_t d = d0 * d0 + d1 * d1 + d2 * d2;
                            if (d < best) { best = d; bi = i; bj = j; bk = k; }
                        }
                uint64_t cell = ((uint64_t)(bi + 1) << 42) ^ ((uint64_t)(bj + 1) << 21) ^ (uint64_t)(bk + 1);
                W->vol[x + W->X * (y + W->Y * z)] = synth_label(W->seed, cell);
            }
}

/* Worley F1 labels: nearest feature point among the 27 cells around the voxel's cell. */
int synth_worley(uint32_t *vol, uint64_t X, uint64_t Y, uint64_t Z, uint32_t cell, uint64_t seed, int n_threads) {
    if (!cell || !X || !Y || !Z) return 1;
    worley_ctx W = {vol, X, Y, Z, seed, (int64_t)cell};
    run_slabs(worley_slab, &W, Z, n_threads);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Fibers (stand-in for the paper's Fiber data set, the stress volume) */
/* ------------------------------------------------------------------ */
/*
 * Tubes along Catmull-Rom splines.  The volume is cut into cells of G^3 voxels;
 * cell (cx, cy, cz) owns T tubes, tube id t = cell * T + k with cell = cx + ncx *
 * (cy + ncy * cz).  A tube has 5 control points: P0 uniform in the cell, then
 * P_i = P_{i-1} + D + J_i per axis (D in [-8, 7] fixed per tube, J_i in [-4, 3]),
 * clamped to the cell box grown by 32 voxels; radius r in {2..6} voxels.  Its
 * two spans (P1 -> P2, P2 -> P3) are sampled at t = q / 16, q = 0..15, as balls
 * of radius r: the centre in 1/8-voxel units is floor(num / 1024) with num =
 * 8192 p1 + 256 A q + 16 B q^2 + C q^3 (A, B, C the Catmull-Rom coefficients:
 * exact integers).  Voxel v (centre 8 v + 4 in those units) belongs to a ball
 * iff sum_a (8 v_a + 4 - c_a)^2 <= (8 r)^2.  A voxel takes the label of the
 * lowest tube id among the balls that hold it (synth_label of that id under
 * seed ^ 0xF1BE5), else 0.  Every ball lies within 48 voxels of its cell box
 * (clamp margin 32, spline overshoot below 5, radius 6), which is what a
 * per-brick generator needs to find the tubes that reach a brick.
 */
#define FIB_BALLS 16
#define FIB_MARGIN 32
#define FIB_REACH 48

static int64_t floor_div(int64_t a, int64_t d) { return a >= 0 ? a / d : -((-a + d - 1) / d); }

static uint64_t fib_hash(uint64_t seed, uint64_t t, uint64_t j) { return hash2(seed ^ 0xF1BE5ull, t * 16 + j); }

static void fib_tube(uint64_t seed, uint64_t t, const int64_t O[3], int64_t G, int64_t P[5][3], int64_t *R) {
    const uint64_t h0 = fib_hash(seed, t, 0), h1 = fib_hash(seed, t, 1);
    int64_t D[3];
    for (int a = 0; a < 3; a++) {
        P[0][a] = O[a] + (int64_t)(((h0 >> (16 * a)) & 0xFFFFull) % (uint64_t)G);
        D[a] = (int64_t)((h1 >> (8 * a)) & 15ull) - 8;
    }
    for (int i = 1; i < 5; i++) {
        const uint64_t h = fib_hash(seed, t, 1 + i);
        for (int a = 0; a < 3; a++) {
            int64_t p = P[i - 1][a] + D[a] + (int64_t)((h >> (8 * a)) & 7ull) - 4;
            const int64_t lo = O[a] - FIB_MARGIN, hi = O[a] + G + FIB_MARGIN - 1;
            P[i][a] = p < lo ? lo : (p > hi ? hi : p);
        }
    }
    *R = 8 * (2 + (int64_t)(fib_hash(seed, t, 6) % 5));
}

static void fib_ball(const int64_t P[5][3], int span, int64_t q, int64_t c[3]) {
    for (int a = 0; a < 3; a++) {
        const int64_t p0 = P[span - 1][a], p1 = P[span][a], p2 = P[span + 1][a], p3 = P[span + 2][a];
        const int64_t A = p2 - p0, B = 2 * p0 - 5 * p1 + 4 * p2 - p3, Cc = -p0 + 3 * p1 - 3 * p2 + p3;
        c[a] = floor_div(8192 * p1 + 256 * A * q + 16 * B * q * q + Cc * q * q * q, 1024);
    }
}

static int64_t isqrt64(int64_t n) {
    int64_t w = (int64_t)sqrt((double)n);
    while (w * w > n) w--;
    while ((w + 1) * (w + 1) <= n) w++;
    return w;
}

/* the whole volume, on the host (small volumes: tests and the oracle's inputs) */
int synth_fibers(uint32_t *vol, uint64_t X, uint64_t Y, uint64_t Z, uint32_t cell, uint32_t tubes, uint64_t seed) {
    if (!vol || !cell || !X || !Y || !Z) return 1;
    const int64_t G = cell, dims[3] = {(int64_t)X, (int64_t)Y, (int64_t)Z};
    const uint64_t ncx = (X + G - 1) / G, ncy = (Y + G - 1) / G, ncz = (Z + G - 1) / G;
    const uint64_t nv = X * Y * Z;
    for (uint64_t i = 0; i < nv; i++) vol[i] = 0xFFFFFFFFu;  /* lowest tube id so far */
    for (uint64_t cz = 0; cz < ncz; cz++)
        for (uint64_t cy = 0; cy < ncy; cy++)
            for (uint64_t cx = 0; cx < ncx; cx++)
                for (uint32_t k = 0; k < tubes; k++) {
                    const uint64_t t = (cx + ncx * (cy + ncy * cz)) * tubes + k;
                    const int64_t O[3] = {(int64_t)cx * G, (int64_t)cy * G, (int64_t)cz * G};
                    int64_t P[5][3], R;
                    fib_tube(seed, t, O, G, P, &R);
                    for (int span = 1; span <= 2; span++)
                        for (int64_t q = 0; q < FIB_BALLS; q++) {
                            int64_t c[3];
                            fib_ball(P, span, q, c);
                            int64_t lo[3], hi[3];
                            for (int a = 0; a < 3; a++) {
                                lo[a] = -floor_div(-(c[a] - 4 - R), 8);  /* ceil */
                                hi[a] = floor_div(c[a] - 4 + R, 8);
                                if (lo[a] < 0) lo[a] = 0;
                                if (hi[a] > dims[a] - 1) hi[a] = dims[a] - 1;
                            }
                            for (int64_t z = lo[2]; z <= hi[2]; z++) {
                                const int64_t dz = 8 * z + 4 - c[2];
                                for (int64_t y = lo[1]; y <= hi[1]; y++) {
                                    const int64_t dy = 8 * y + 4 - c[1], rem = R * R - dz * dz - dy * dy;
                                    if (rem < 0) continue;
                                    const int64_t w = isqrt64(rem);
                                    int64_t x0 = -floor_div(-(c[0] - 4 - w), 8), x1 = floor_div(c[0] - 4 + w, 8);
                                    if (x0 < lo[0]) x0 = lo[0];
                                    if (x1 > hi[0]) x1 = hi[0];
                                    uint32_t *row = vol + (uint64_t)y * X + (uint64_t)z * X * Y;
                                    for (int64_t x = x0; x <= x1; x++)
                                        if ((uint32_t)t < row[x]) row[x] = (uint32_t)t;
                                }
                            }
                        }
                }
    for (uint64_t i = 0; i < nv; i++) vol[i] = vol[i] == 0xFFFFFFFFu ? 0u : synth_label(seed ^ 0xF1BE5ull, vol[i]);
    return 0;
}
