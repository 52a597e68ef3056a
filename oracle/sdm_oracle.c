/*
 * Plain, slow CPU oracle of the Super-Droplet Method (SDM) collision-coalescence
 * step.  TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  The
 * product path (the CUDA library) never does, and the two share no source.
 *
 * What it computes (paper: Introduction, which names Shima et al.'s (2009)
 * Monte-Carlo SDM scheme as the model of collisional growth; API in brief, the
 * Box(dt, dv) + Coalescence(Golovin(b)) example; Usage examples, Box
 * environment, the Golovin and Berry geometric sweep-out kernels).  The paper
 * names the algorithm but prints no formulae; the step below follows the
 * four-part statement of the method this library implements:
 *
 *   1. per cell, a random permutation of the live super-droplets (SDs):
 *      sort by a 64-bit random key, ties by rank;
 *   2. neighbours in the permuted list form floor(n_c/2) candidate pairs;
 *   3. p = K(j,k) * max(xi_j, xi_k) * dt/dV * [n_c(n_c-1)/2] / floor(n_c/2),
 *      gamma = ceil(p - u), u ~ U[0,1), capped at floor(xi_j/xi_k);
 *   4. Shima update: xi_j -= gamma*xi_k with v_k += gamma*v_j, or, when that
 *      leaves xi_j at zero, a split of the k SD into two halves; an SD whose
 *      multiplicity reaches zero is dead and drops out of later steps.
 *
 * Every free choice (random-number layout, tie-breaks, cube root, operation
 * order) is fixed here so that a second implementation can reproduce the
 * result bit for bit.  All floating point is IEEE binary64/binary32 with
 * round-to-nearest and no contraction: build with -ffp-contract=off.
 *
 * Sedimentation (a next step of the method, paper: API in brief, the
 * displacement of particles among the listed dynamics; Usage examples, the 2-D example's
 * sedimenting drizzle): every live SD falls by its Rogers-Yau fall speed
 * times dt.  Cells are levels x columns (cell = iz * nx + ix, levels of
 * height dz); an SD's position is its height zeta above its cell's bottom.
 * SDs falling through the bottom leave the domain (cell -1: outside, never
 * stepped) and their water is precipitated; dead SDs leave it as well.
 *
 * Parity status: every function below is pinned by tests/test_oracle_*.py
 * (Philox known answers, hand-worked Shima pairs, brute-force pairing and
 * gamma frequencies in both precisions, binary32 hand cases of p, volume
 * conservation, the Golovin closed form, hand-worked per-cell spectra).  The
 * geometric (Rogers-Yau) kernel has no closed form; it is pinned by
 * invariants only (symmetry, K(r,r) = 0, regime values, conservation).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

typedef struct {
    int32_t kernel;    /* 0: Golovin additive, 1: geometric sweep-out (Rogers-Yau v_t),
                          2: geometric sweep-out times Long's (1974) collision efficiency */
    int32_t precision; /* 0: K and p in binary64; 1: K and p in binary32 */
    double b;          /* Golovin constant, s^-1 */
    double dt;         /* timestep, s */
    double dv;         /* cell volume, m^3 */
    double k1, k2, k3; /* Rogers-Yau: k1 r^2 | k2 r | k3 sqrt(r) (SI) */
    double r1, r2;     /* Rogers-Yau regime bounds, m */
    uint64_t seed;     /* Philox key of instance 0; instance i uses seed + i */
} orc_params;

typedef struct {
    int64_t n_pairs;      /* candidate pairs examined */
    int64_t n_collisions; /* pairs with gamma > 0 */
    int64_t sum_gamma;    /* sum of gamma over all pairs */
} orc_stats;

/* ------------------------------------------------------------------ Philox */
/* Philox4x32-10 of Salmon, Moraes, Dror & Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplies with
 * the Weyl key schedule. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ x1 ^ k0;
        uint32_t n2 = hi0 ^ x3 ^ k1;
        x0 = n0;
        x1 = lo1;
        x2 = n2;
        x3 = lo0;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

/* Counter layout (the paper is silent on random-number streams).
 *   key   = (low 32 bits of the instance seed, high 32 bits)
 *   ctr   = (index >> 1, cell, low 32 bits of s, (high 31 bits of s) | tag << 31)
 * tag 0 draws the sort key of the SD of rank `index` in the cell, tag 1 the
 * uniform number of candidate pair `index`; the even index takes output
 * words (0, 1), the odd index words (2, 3). */
static void draw_two_words(uint64_t seed, uint32_t index, uint32_t cell, int64_t s, uint32_t tag,
                           uint32_t *wa, uint32_t *wb)
{
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = index >> 1;
    ctr[1] = cell;
    ctr[2] = (uint32_t)((uint64_t)s & 0xFFFFFFFFu);
    ctr[3] = ((uint32_t)((uint64_t)s >> 32) & 0x7FFFFFFFu) | (tag << 31);
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
    orc_philox4x32_10(ctr, key, out);
    if (index & 1u) {
        *wa = out[2];
        *wb = out[3];
    } else {
        *wa = out[0];
        *wb = out[1];
    }
}

uint64_t orc_sort_key(uint64_t seed, uint32_t rank, uint32_t cell, int64_t s)
{
    uint32_t wa, wb;
    draw_two_words(seed, rank, cell, s, 0u, &wa, &wb);
    return ((uint64_t)wa << 32) | (uint64_t)wb;
}

/* u = m * 2^-53 with m the 53-bit integer (wa << 21) | (wb >> 11): exact, in [0, 1). */
double orc_pair_uniform(uint64_t seed, uint32_t pair, uint32_t cell, int64_t s)
{
    uint32_t wa, wb;
    draw_two_words(seed, pair, cell, s, 1u, &wa, &wb);
    uint64_t m = ((uint64_t)wa << 21) | (uint64_t)(wb >> 11);
    return (double)m * 0x1p-53;
}

/* --------------------------------------------------------------- cube root */
/* r = (3 v / 4 pi)^(1/3) needs a cube root that two implementations can
 * reproduce exactly, so it is defined here as a fixed sequence of IEEE basic
 * operations: split x = f 2^E (f in [1,2)), E = 3k + j (j in 0..2), m = f 2^j;
 * a quadratic seed for m^(-1/3) refined by two Newton steps for the inverse
 * cube root in binary32; then two binary64 corrections
 * y <- y - (y*y*y - m) * R with R = 1/(3 y^2) taken from the binary32 stage;
 * finally y 2^k.  Accurate to 1 ulp of binary64 (pinned against libm). */
static const float CBRT_P0 = 0x1.610e12p+0f;   /* quadratic fit of f^(-1/3), f in [1,2) */
static const float CBRT_P1 = -0x1.e43e5cp-2f;
static const float CBRT_P2 = 0x1.72f4a4p-4f;
static const float CBRT_THIRD = 0x1.555556p-2f; /* 1/3 rounded to binary32 */
static const float CBRT_C[3] = {1.0f, 0x1.965feap-1f, 0x1.428a30p-1f}; /* 2^(-j/3) */

static double pow2_int(int e) /* exact 2^e for -1022 <= e <= 1023 */
{
    uint64_t bits = (uint64_t)(e + 1023) << 52;
    double d;
    memcpy(&d, &bits, sizeof d);
    return d;
}

static float inv_cbrt_seed(float ff, float mf, int j)
{
    float z = CBRT_P2 * ff;
    z = CBRT_P1 + z;
    z = ff * z;
    z = CBRT_P0 + z;
    z = z * CBRT_C[j];
    for (int it = 0; it < 2; ++it) {
        float t = z * z;
        t = t * z;
        t = mf * t;
        t = 1.0f - t;
        t = t * z;
        t = t * CBRT_THIRD;
        z = z + t;
    }
    return z;
}

/* x: positive normal binary64. */
double orc_cbrt(double x)
{
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    int E = (int)((bits >> 52) & 0x7FF) - 1023;
    int k = (E + 3069) / 3 - 1023; /* floor(E / 3) */
    int j = E - 3 * k;
    uint64_t fbits = (bits & 0x000FFFFFFFFFFFFFull) | ((uint64_t)1023 << 52);
    double f;
    memcpy(&f, &fbits, sizeof f);
    double m = f * pow2_int(j);
    float ff = (float)f;
    float mf = (float)m;
    float z = inv_cbrt_seed(ff, mf, j);
    float zz = z * z;
    float yf = mf * zz;
    float rf = zz * CBRT_THIRD;
    double y = (double)yf;
    double R = (double)rf;
    for (int it = 0; it < 2; ++it) {
        double c = y * y;
        c = c * y;
        c = c - m;
        c = c * R;
        y = y - c;
    }
    return y * pow2_int(k);
}

static float pow2f_int(int e) /* exact 2^e for -126 <= e <= 127 */
{
    uint32_t bits = (uint32_t)(e + 127) << 23;
    float f;
    memcpy(&f, &bits, sizeof f);
    return f;
}

/* binary32 twin (same seed and inverse-cube-root steps, one binary32
 * correction instead of two binary64 ones).  x: positive normal binary32. */
float orc_cbrtf(float x)
{
    uint32_t bits;
    memcpy(&bits, &x, sizeof bits);
    int E = (int)((bits >> 23) & 0xFF) - 127;
    int k = (E + 381) / 3 - 127; /* floor(E / 3) */
    int j = E - 3 * k;
    uint32_t fbits = (bits & 0x007FFFFFu) | (127u << 23);
    float ff;
    memcpy(&ff, &fbits, sizeof ff);
    float mf = ff * pow2f_int(j);
    float z = inv_cbrt_seed(ff, mf, j);
    float zz = z * z;
    float yf = mf * zz;
    float rf = zz * CBRT_THIRD;
    float c = yf * yf;
    c = c * yf;
    c = c - mf;
    c = c * rf;
    yf = yf - c;
    return yf * pow2f_int(k);
}

/* ------------------------------------------------------- collision kernels */
static const double ORC_PI = 3.141592653589793;

double orc_radius(double v) { return orc_cbrt(v * (0.75 / ORC_PI)); }

float orc_radiusf(float v) { return orc_cbrtf(v * (float)(0.75 / ORC_PI)); }

/* Rogers & Yau (1989) piecewise terminal velocity. */
double orc_vt(const orc_params *P, double r)
{
    if (r < P->r1)
        return P->k1 * (r * r);
    if (r < P->r2)
        return P->k2 * r;
    return P->k3 * sqrt(r);
}

float orc_vtf(const orc_params *P, float r)
{
    if (r < (float)P->r1)
        return (float)P->k1 * (r * r);
    if (r < (float)P->r2)
        return (float)P->k2 * r;
    return (float)P->k3 * sqrtf(r);
}

/* Collision efficiency of Long (1974, J. Atmos. Sci. 31, 1040-1052), the
 * form later SDM studies use for their hydrodynamic ("Long") kernel: with
 * R the larger and r the smaller radius of the pair,
 *   E = max(c1 R^2 (1 - c2 / r), E_min)   for R <= R_lim,
 *   E = 1                                 for R >  R_lim,
 * c1 = 4.5e4 cm^-2 = 4.5e8 m^-2, c2 = 3e-4 cm = 3e-6 m, E_min = 1e-3,
 * R_lim = 50 um.  (The form reaches 1.0575 at R = r = 50 um; it is used as
 * published, without a cap at 1.)  Binary64, in this operation order. */
double orc_efficiency_long(double rj, double rk)
{
    double R = rj > rk ? rj : rk;
    double r = rj > rk ? rk : rj;
    if (R > 50e-6)
        return 1.0;
    double e = (4.5e8 * (R * R)) * (1.0 - 3e-6 / r);
    return e < 1e-3 ? 1e-3 : e;
}

/* The same in binary32, with the binary32 roundings of the binary64
 * constants. */
float orc_efficiency_longf(float rj, float rk)
{
    float R = rj > rk ? rj : rk;
    float r = rj > rk ? rk : rj;
    if (R > (float)50e-6)
        return 1.0f;
    float e = ((float)4.5e8 * (R * R)) * (1.0f - (float)3e-6 / r);
    return e < (float)1e-3 ? (float)1e-3 : e;
}

/* K(j,k) in m^3 s^-1: Golovin b (v_j + v_k) (kernel 0); geometric sweep-out
 * pi (r_j + r_k)^2 |v_t(r_j) - v_t(r_k)| with collection efficiency 1
 * (kernel 1); the same sweep-out times Long's efficiency E(r_j, r_k)
 * (kernel 2). */
double orc_kernel(const orc_params *P, double vj, double vk)
{
    if (P->kernel == 0)
        return P->b * (vj + vk);
    double rj = orc_radius(vj), rk = orc_radius(vk);
    double s = rj + rk;
    double K = (ORC_PI * (s * s)) * fabs(orc_vt(P, rj) - orc_vt(P, rk));
    if (P->kernel == 2)
        K = K * orc_efficiency_long(rj, rk);
    return K;
}

float orc_kernelf(const orc_params *P, float vj, float vk)
{
    if (P->kernel == 0)
        return (float)P->b * (vj + vk);
    float rj = orc_radiusf(vj), rk = orc_radiusf(vk);
    float s = rj + rk;
    float K = ((float)ORC_PI * (s * s)) * fabsf(orc_vtf(P, rj) - orc_vtf(P, rk));
    if (P->kernel == 2)
        K = K * orc_efficiency_longf(rj, rk);
    return K;
}

/* dt/dV * [n_c(n_c-1)/2] / floor(n_c/2): the factor that rescales the pair
 * probability from the n_c(n_c-1)/2 possible pairs to the floor(n_c/2) drawn. */
double orc_scale(const orc_params *P, int64_t n_c)
{
    double dtdv = P->dt / P->dv;
    double ratio = (double)(n_c * (n_c - 1) / 2) / (double)(n_c / 2);
    return dtdv * ratio;
}

/* p for the pair (j, k), xi_j >= xi_k. */
double orc_probability(const orc_params *P, double scale, int64_t xi_j, double vj, double vk)
{
    if (P->precision == 0) {
        double K = orc_kernel(P, vj, vk);
        return (K * (double)xi_j) * scale;
    }
    float Kf = orc_kernelf(P, (float)vj, (float)vk);
    float pf = (Kf * (float)xi_j) * (float)scale;
    return (double)pf;
}

/* gamma = ceil(p - u) capped at floor(xi_j / xi_k), compared in binary64
 * before the integer conversion so that a huge p cannot overflow. */
int64_t orc_gamma(double p, double u, int64_t xi_j, int64_t xi_k)
{
    double g = ceil(p - u);
    int64_t q = xi_j / xi_k;
    if (g >= (double)q)
        return q;
    return (int64_t)g;
}

/* Shima update of one pair for gamma collisions; xi_j >= xi_k > 0. */
void orc_update(int64_t gamma, int64_t *xi_j, int64_t *xi_k, double *vj, double *vk)
{
    if (gamma == 0)
        return;
    double t = (double)gamma * *vj;
    double vnew = *vk + t;
    int64_t rem = *xi_j - gamma * *xi_k;
    if (rem > 0) {
        *xi_j = rem;
        *vk = vnew;
    } else {
        int64_t h = *xi_k / 2;
        *xi_j = h;
        *xi_k = *xi_k - h;
        *vj = vnew;
        *vk = vnew;
    }
}

/* ------------------------------------------------------------------ a step */
typedef struct {
    uint64_t key;
    uint32_t rank;
    int64_t sd; /* index into the caller's arrays */
} live_entry;

static int cmp_live(const void *a, const void *b)
{
    const live_entry *x = (const live_entry *)a, *y = (const live_entry *)b;
    if (x->key != y->key)
        return x->key < y->key ? -1 : 1;
    if (x->rank != y->rank)
        return x->rank < y->rank ? -1 : 1;
    return 0;
}

/* The total order of the permutation, exposed for tests: <0, 0, >0. */
int orc_order(uint64_t key_a, uint32_t rank_a, uint64_t key_b, uint32_t rank_b)
{
    live_entry a = {key_a, rank_a, 0}, b = {key_b, rank_b, 0};
    return cmp_live(&a, &b);
}

/* Group SDs by (instance, cell); members listed in increasing SD index, so
 * that the position within the group is the SD's rank.  Returns group start
 * offsets (n_groups + 1) and the member list. */
static int group_sds(int64_t n_sd, int32_t n_cells, int32_t n_inst, const int32_t *cell,
                     const int32_t *inst, int64_t **start_out, int64_t **members_out)
{
    int64_t n_groups = (int64_t)n_cells * n_inst;
    int64_t *start = (int64_t *)calloc((size_t)n_groups + 1, sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)n_groups + 1, sizeof(int64_t));
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_sd > 0 ? n_sd : 1));
    if (!start || !fill || !members) {
        free(start);
        free(fill);
        free(members);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < n_sd; ++i) {
        if (cell[i] < 0)
            continue; /* outside the domain */
        int64_t g = (int64_t)(inst ? inst[i] : 0) * n_cells + cell[i];
        start[g + 1] += 1;
    }
    for (int64_t g = 0; g < n_groups; ++g)
        start[g + 1] += start[g];
    for (int64_t i = 0; i < n_sd; ++i) {
        if (cell[i] < 0)
            continue;
        int64_t g = (int64_t)(inst ? inst[i] : 0) * n_cells + cell[i];
        members[start[g] + fill[g]] = i;
        fill[g] += 1;
    }
    free(fill);
    *start_out = start;
    *members_out = members;
    return ORC_OK;
}

static int check_layout(int64_t n_sd, int32_t n_cells, int32_t n_inst, const int32_t *cell,
                        const int32_t *inst)
{
    if (n_sd < 0 || n_cells < 1 || n_inst < 1)
        return ORC_EINVAL;
    for (int64_t i = 0; i < n_sd; ++i) {
        if (cell[i] < -1 || cell[i] >= n_cells) /* -1: outside the domain */
            return ORC_EINVAL;
        if (inst && (inst[i] < 0 || inst[i] >= n_inst))
            return ORC_EINVAL;
    }
    return ORC_OK;
}

/* The random permutation of one cell: the live SDs (xi > 0) among the n
 * members given in rank order, sorted by (sort key, rank).  Writes the ranks
 * in permuted order to perm[0 .. n_c) and returns n_c.  `scratch` holds n
 * entries. */
static int64_t permute_cell(uint64_t seed, uint32_t c, int64_t s, const int64_t *xi_members,
                            int64_t n, live_entry *scratch)
{
    int64_t n_c = 0;
    for (int64_t q = 0; q < n; ++q) {
        if (xi_members[q] > 0) {
            scratch[n_c].key = orc_sort_key(seed, (uint32_t)q, c, s);
            scratch[n_c].rank = (uint32_t)q;
            scratch[n_c].sd = q;
            n_c += 1;
        }
    }
    qsort(scratch, (size_t)n_c, sizeof(live_entry), cmp_live);
    return n_c;
}

int64_t orc_permutation(uint64_t seed, uint32_t cell, int64_t s, const int64_t *xi_members,
                        int64_t n, int64_t *perm)
{
    live_entry *L = (live_entry *)malloc(sizeof(live_entry) * (size_t)(n > 0 ? n : 1));
    if (!L)
        return -1;
    int64_t n_c = permute_cell(seed, cell, s, xi_members, n, L);
    for (int64_t q = 0; q < n_c; ++q)
        perm[q] = (int64_t)L[q].rank;
    free(L);
    return n_c;
}

/* One coalescence step with global step index s over every cell of every
 * instance.  xi and v are updated in place; they are indexed by SD id. */
int orc_step(const orc_params *P, int64_t n_sd, int32_t n_cells, int32_t n_inst,
             const int32_t *cell, const int32_t *inst, int64_t *xi, double *v, int64_t s,
             orc_stats *st)
{
    int rc = check_layout(n_sd, n_cells, n_inst, cell, inst);
    if (rc != ORC_OK)
        return rc;
    if (s < 0)
        return ORC_EINVAL;
    int64_t *start, *members;
    rc = group_sds(n_sd, n_cells, n_inst, cell, inst, &start, &members);
    if (rc != ORC_OK)
        return rc;
    int64_t max_group = 0;
    int64_t n_groups = (int64_t)n_cells * n_inst;
    for (int64_t g = 0; g < n_groups; ++g)
        if (start[g + 1] - start[g] > max_group)
            max_group = start[g + 1] - start[g];
    size_t cap = (size_t)(max_group > 0 ? max_group : 1);
    live_entry *L = (live_entry *)malloc(sizeof(live_entry) * cap);
    int64_t *xm = (int64_t *)malloc(sizeof(int64_t) * cap);
    if (!L || !xm) {
        free(L);
        free(xm);
        free(start);
        free(members);
        return ORC_ENOMEM;
    }
    int64_t pairs = 0, colls = 0, gsum = 0;
    for (int64_t g = 0; g < n_groups; ++g) {
        uint32_t c = (uint32_t)(g % n_cells);
        uint64_t seed = P->seed + (uint64_t)(g / n_cells);
        int64_t n = start[g + 1] - start[g];
        const int64_t *mem = members + start[g];
        for (int64_t q = 0; q < n; ++q)
            xm[q] = xi[mem[q]];
        /* 1. the random permutation of the live SDs */
        int64_t n_c = permute_cell(seed, c, s, xm, n, L);
        if (n_c < 2)
            continue;
        /* 2. pairs of neighbours; 3. probability and collision count */
        double scale = orc_scale(P, n_c);
        for (int64_t l = 0; l < n_c / 2; ++l) {
            int64_t a = mem[L[2 * l].sd], b = mem[L[2 * l + 1].sd];
            int64_t j = a, k = b;
            if (xi[a] < xi[b]) {
                j = b;
                k = a;
            }
            double p = orc_probability(P, scale, xi[j], v[j], v[k]);
            double u = orc_pair_uniform(seed, (uint32_t)l, c, s);
            int64_t gamma = orc_gamma(p, u, xi[j], xi[k]);
            /* 4. Shima update */
            orc_update(gamma, &xi[j], &xi[k], &v[j], &v[k]);
            pairs += 1;
            colls += gamma > 0;
            gsum += gamma;
        }
    }
    free(L);
    free(xm);
    free(start);
    free(members);
    if (st) {
        st->n_pairs += pairs;
        st->n_collisions += colls;
        st->sum_gamma += gsum;
    }
    return ORC_OK;
}

/* n_steps consecutive steps with indices s0, s0+1, ... */
int orc_run(const orc_params *P, int64_t n_sd, int32_t n_cells, int32_t n_inst,
            const int32_t *cell, const int32_t *inst, int64_t *xi, double *v, int64_t s0,
            int64_t n_steps, orc_stats *st)
{
    for (int64_t t = 0; t < n_steps; ++t) {
        int rc = orc_step(P, n_sd, n_cells, n_inst, cell, inst, xi, v, s0 + t, st);
        if (rc != ORC_OK)
            return rc;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------- spectrum */
/* The ParticlesVolumeSpectrum product dv/dlnr (paper: API in brief): per
 * radius bin [e_b, e_{b+1}) the volume of live SDs, sum(xi v), per unit
 * volume of air and per unit ln r.  per_cell != 0: out[g * n_bins + b] for
 * group g = instance * n_cells + cell, normalised by dv; otherwise out[b]
 * over all cells, normalised by dv * n_cells * n_inst.  Sums run in SD-index
 * order. */
int orc_spectrum(const orc_params *P, int64_t n_sd, int32_t n_cells, int32_t n_inst,
                 const int32_t *cell, const int32_t *inst, const int64_t *xi, const double *v,
                 const double *edges, int32_t n_edges, int32_t per_cell, double *out)
{
    int rc = check_layout(n_sd, n_cells, n_inst, cell, inst);
    if (rc != ORC_OK)
        return rc;
    if (n_edges < 2)
        return ORC_EINVAL;
    for (int32_t e = 0; e + 1 < n_edges; ++e)
        if (!(edges[e] > 0.0) || !(edges[e + 1] > edges[e]))
            return ORC_EINVAL;
    int32_t n_bins = n_edges - 1;
    int64_t n_out = per_cell ? (int64_t)n_cells * n_inst * n_bins : n_bins;
    for (int64_t q = 0; q < n_out; ++q)
        out[q] = 0.0;
    for (int64_t i = 0; i < n_sd; ++i) {
        if (xi[i] <= 0 || cell[i] < 0)
            continue;
        double r = orc_radius(v[i]);
        if (r < edges[0] || !(r < edges[n_edges - 1]))
            continue;
        int32_t lo = 0, hi = n_edges - 1; /* edges[lo] <= r < edges[hi] */
        while (hi - lo > 1) {
            int32_t mid = (lo + hi) / 2;
            if (edges[mid] <= r)
                lo = mid;
            else
                hi = mid;
        }
        int64_t g = (int64_t)(inst ? inst[i] : 0) * n_cells + cell[i];
        int64_t slot = per_cell ? g * n_bins + lo : lo;
        out[slot] += (double)xi[i] * v[i];
    }
    double vol = per_cell ? P->dv : P->dv * (double)n_cells * (double)n_inst;
    for (int64_t q = 0; q < n_out; ++q) {
        int32_t bin = (int32_t)(q % n_bins);
        out[q] = out[q] / vol / (log(edges[bin + 1]) - log(edges[bin]));
    }
    return ORC_OK;
}

/* ------------------------------------------------------------ sedimentation */
/* The fall of one SD in one step: its height zeta above the bottom of level
 * iz drops by d; each time it goes below zero the SD enters the level below,
 * whose top it reaches with zeta + dz.  Returns the new level (-1: through
 * the bottom of the domain) and writes the new zeta.  If zeta + dz rounds up
 * to dz itself, the SD is on the boundary and stays in the level above, at
 * zeta = 0 (levels are half-open [iz dz, (iz + 1) dz)). */
int32_t orc_fall(double zeta, int32_t iz, double d, double dz, double *zeta_out)
{
    double z = zeta - d;
    while (z < 0.0) {
        iz -= 1;
        if (iz < 0) {
            *zeta_out = 0.0;
            return -1;
        }
        z = z + dz;
    }
    if (z >= dz) {
        iz += 1;
        z = 0.0;
    }
    *zeta_out = z;
    return iz;
}

/* The fall distance of one step: the Rogers-Yau speed of the binary32
 * radius twin, times dt, in binary32 (the speed formula itself is good to
 * some per cent), widened exactly to binary64. */
double orc_fall_distance(const orc_params *P, double v)
{
    float r = orc_radiusf((float)v);
    float vt = orc_vtf(P, r);
    return (double)(vt * (float)P->dt);
}

/* One sedimentation step over every SD, in SD-id order.  cell, zeta are
 * updated in place; *precip (if given) is increased by xi v of every SD that
 * falls through the bottom (summed in id order).  Dead SDs (xi = 0) and SDs
 * already outside end up outside (cell -1, zeta 0). */
int orc_sediment(const orc_params *P, int64_t n_sd, int32_t nx, int32_t n_cells, double dz,
                 const int64_t *xi, const double *v, int32_t *cell, double *zeta, double *precip)
{
    if (nx < 1 || n_cells % nx != 0 || !(dz > 0.0))
        return ORC_EINVAL;
    int rc = check_layout(n_sd, n_cells, 1, cell, NULL);
    if (rc != ORC_OK)
        return rc;
    for (int64_t i = 0; i < n_sd; ++i) {
        if (cell[i] < 0 || xi[i] <= 0) {
            cell[i] = -1;
            zeta[i] = 0.0;
            continue;
        }
        int32_t iz = cell[i] / nx, ix = cell[i] % nx;
        double d = orc_fall_distance(P, v[i]);
        iz = orc_fall(zeta[i], iz, d, dz, &zeta[i]);
        if (iz < 0) {
            if (precip)
                *precip += (double)xi[i] * v[i];
            cell[i] = -1;
            continue;
        }
        cell[i] = iz * nx + ix;
    }
    return ORC_OK;
}

/* Height above the cell's bottom from the height above the domain bottom,
 * and back: zeta = z - iz dz, z = iz dz + zeta (binary64, each product and
 * sum rounded once). */
double orc_zeta_of(double z, int32_t cell, int32_t nx, double dz) { return z - (double)(cell / nx) * dz; }

double orc_z_of(double zeta, int32_t cell, int32_t nx, double dz) { return (double)(cell / nx) * dz + zeta; }

/* ------------------------------------------------------------- condensation */
/* Diffusional growth of every live SD inside the domain over one step, in
 * the large-drop limit of the growth law r dr/dt = s G (Rogers & Yau 1989,
 * ch. 7, with the curvature and solute terms dropped): s is the cell's
 * supersaturation (S - 1) and G = 1 / (F_k + F_d) its growth coefficient,
 * m^2 s^-1, both held over the step, so r^2 grows by exactly
 * c = 2 G s dt.  An evaporating SD stops at the floor radius r_min, or at
 * its own radius when that is already below r_min.
 *
 * Reading (as for the fall distance): the change of volume is evaluated in
 * binary32, from the binary32 image of the volume and its binary32 radius,
 * as the difference of (4 pi / 3) x^(3/2) at x' = x + c and at x = r^2,
 * written without cancellation,
 *   dV = k43 (d ((x' + a b) + x)) / (a + b),  a = sqrt(x'), b = sqrt(x),
 * with d = x' - x taken as c itself (not as the rounded difference, which
 * would lose the digits of c below x's last bit) unless the floor acts, and
 * then as floor - x; dV is widened exactly and added to the binary64
 * volume.  Multiplicities do not
 * change.  condensed (nullable, n_cells entries) receives sum(xi dV) of
 * each cell, m^3 (summed in SD-id order). */
int orc_condense(const orc_params *P, int64_t n_sd, int32_t n_cells, const int32_t *cell, const int64_t *xi,
                 double *v, const double *G, const double *s, double r_min, double *condensed)
{
    int rc = check_layout(n_sd, n_cells, 1, cell, NULL);
    if (rc != ORC_OK)
        return rc;
    if (!(r_min > 0.0))
        return ORC_EINVAL;
    if (condensed)
        for (int32_t c = 0; c < n_cells; ++c)
            condensed[c] = 0.0;
    const float k43 = (float)(4.0 * ORC_PI / 3.0);
    const float xmin = (float)(r_min * r_min);
    for (int64_t i = 0; i < n_sd; ++i) {
        int32_t c = cell[i];
        if (c < 0 || xi[i] <= 0)
            continue;
        float cf = (float)(((2.0 * G[c]) * s[c]) * P->dt);
        float r = orc_radiusf((float)v[i]);
        float x = r * r;
        float xn = x + cf;
        float lo = x < xmin ? x : xmin;
        float d = cf; /* x' - x, exact where the floor does not act */
        if (xn < lo) {
            xn = lo;
            d = lo - x;
        }
        float dv = 0.0f;
        if (d != 0.0f) {
            float a = sqrtf(xn), b = sqrtf(x);
            dv = k43 * ((d * ((xn + a * b) + x)) / (a + b));
        }
        v[i] = v[i] + (double)dv;
        if (condensed)
            condensed[c] += (double)xi[i] * (double)dv;
    }
    return ORC_OK;
}
