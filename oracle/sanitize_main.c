/*
 * Driver that runs every entry point of the CPU oracle on ragged inputs, for
 * a build under AddressSanitizer and UndefinedBehaviorSanitizer (test
 * infrastructure only; tests/test_oracle_sanitized.py builds and runs it).
 * The oracle's source is included whole, so the driver sees its types.
 *
 * Cases: layouts of 1 to 37 cells in 1 or 2 instances with empty, single-SD
 * and large cells, dead SDs, multiplicities up to 2^62, SDs outside the
 * domain, all three collision kernels in both precisions, p far below and far
 * above 1; total and per-cell spectra; sedimentation steps; the permutation
 * and the pair-level functions; and rejected layouts.  Exits non-zero on an
 * unexpected status or a broken conservation law (sum xi v kept to 1e-12,
 * sum xi never rising).
 */
#include "sdm_oracle.c"

#include <stdio.h>

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;

static uint64_t next_u64(void) /* xorshift64* */
{
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return rng_state * 0x2545F4914F6CDD1Dull;
}

static double next_unit(void) { return (double)(next_u64() >> 11) * 0x1p-53; }

static int failures = 0;

static void expect(int ok, const char *what, int case_id)
{
    if (!ok) {
        fprintf(stderr, "case %d: %s\n", case_id, what);
        ++failures;
    }
}

static void run_case(int case_id, int32_t n_cells, int32_t n_inst, int32_t max_per_cell, int32_t kernel,
                     int32_t precision, double dv, int huge_xi)
{
    int64_t n_sd = 0;
    int32_t *count = (int32_t *)calloc((size_t)n_cells * (size_t)n_inst, sizeof(int32_t));
    for (int32_t g = 0; g < n_cells * n_inst; ++g) {
        const uint64_t r = next_u64() % 10u;
        count[g] = r == 0 ? 0 : r == 1 ? 1 : (int32_t)(next_u64() % (uint64_t)(max_per_cell + 1));
        n_sd += count[g];
    }
    const int64_t n_out = 3; /* SDs outside the domain */
    const int64_t n = n_sd + n_out;
    int32_t *cell = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *inst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *xi = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double *v = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *zeta = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int64_t i = 0;
    for (int32_t g = 0; g < n_cells * n_inst; ++g)
        for (int32_t k = 0; k < count[g]; ++k, ++i) {
            cell[i] = g % n_cells;
            inst[i] = g / n_cells;
        }
    for (; i < n; ++i) {
        cell[i] = -1;
        inst[i] = 0;
    }
    /* shuffle the SD order (ids are positions) */
    for (int64_t a = n - 1; a > 0; --a) {
        const int64_t b = (int64_t)(next_u64() % (uint64_t)(a + 1));
        const int32_t tc = cell[a], ti = inst[a];
        cell[a] = cell[b];
        inst[a] = inst[b];
        cell[b] = tc;
        inst[b] = ti;
    }
    for (i = 0; i < n; ++i) {
        const uint64_t r = next_u64() % 20u;
        xi[i] = r == 0 ? 0 : r == 1 ? 1 : (huge_xi && r == 2) ? ((int64_t)1 << 62) : (int64_t)(1 + next_u64() % 1000000000u);
        const double rad = exp(log(2e-6) + next_unit() * (log(2e-3) - log(2e-6)));
        v[i] = 4.0 / 3.0 * ORC_PI * rad * rad * rad;
        zeta[i] = next_unit() * 10.0;
    }

    orc_params P;
    P.kernel = kernel;
    P.precision = precision;
    P.b = 1500.0;
    P.dt = 1.0;
    P.dv = dv;
    P.k1 = 1.19e8;
    P.k2 = 8e3;
    P.k3 = 201.0;
    P.r1 = 40e-6;
    P.r2 = 600e-6;
    P.seed = next_u64();

    long double w0 = 0.0L, x0 = 0.0L;
    for (i = 0; i < n; ++i)
        if (cell[i] >= 0) {
            w0 += (long double)xi[i] * (long double)v[i];
            x0 += (long double)xi[i];
        }
    orc_stats st = {0, 0, 0};
    expect(orc_run(&P, n, n_cells, n_inst, cell, inst, xi, v, 5, 25, &st) == ORC_OK, "run", case_id);
    long double w1 = 0.0L, x1 = 0.0L;
    for (i = 0; i < n; ++i)
        if (cell[i] >= 0) {
            w1 += (long double)xi[i] * (long double)v[i];
            x1 += (long double)xi[i];
            expect(xi[i] >= 0, "negative multiplicity", case_id);
        }
    expect(x1 <= x0, "sum xi rose", case_id);
    expect(fabsl(w1 - w0) <= 1e-12L * (w0 > 0 ? w0 : 1.0L), "sum xi v not conserved", case_id);

    double edges[33];
    for (int e = 0; e < 33; ++e)
        edges[e] = 1e-5 * pow(500.0, e / 32.0);
    double *spec = (double *)malloc(sizeof(double) * (size_t)n_cells * (size_t)n_inst * 32u);
    expect(orc_spectrum(&P, n, n_cells, n_inst, cell, inst, xi, v, edges, 33, 0, spec) == ORC_OK, "spectrum",
           case_id);
    expect(orc_spectrum(&P, n, n_cells, n_inst, cell, inst, xi, v, edges, 33, 1, spec) == ORC_OK,
           "per-cell spectrum", case_id);
    edges[5] = edges[4]; /* not increasing: rejected */
    expect(orc_spectrum(&P, n, n_cells, n_inst, cell, inst, xi, v, edges, 33, 0, spec) == ORC_EINVAL,
           "bad edges accepted", case_id);

    if (n_inst == 1) {
        double precip = 0.0;
        const int32_t nx = n_cells % 2 == 0 ? 2 : 1;
        for (int t = 0; t < 4; ++t)
            expect(orc_sediment(&P, n, nx, n_cells, 10.0, xi, v, cell, zeta, &precip) == ORC_OK, "sediment",
                   case_id);
        expect(precip >= 0.0, "negative precipitation", case_id);
        expect(orc_sediment(&P, n, 3, n_cells * 3 + 1, 10.0, xi, v, cell, zeta, &precip) == ORC_EINVAL,
               "bad column count accepted", case_id);
    }

    /* permutation of cell 0 of instance 0, into arrays of exactly its size */
    int64_t m = 0;
    for (i = 0; i < n; ++i)
        m += cell[i] == 0 && inst[i] == 0;
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    m = 0;
    for (i = 0; i < n; ++i)
        if (cell[i] == 0 && inst[i] == 0)
            members[m++] = xi[i];
    const int64_t n_c = orc_permutation(P.seed, 0, 7, members, m, perm);
    expect(n_c >= 0 && n_c <= m, "permutation count", case_id);
    for (int64_t q = 0; q < n_c; ++q)
        expect(perm[q] >= 0 && perm[q] < m, "permutation rank", case_id);

    /* a layout with a cell id out of range is rejected before any work */
    if (n > 0) {
        const int32_t keep = cell[0];
        cell[0] = n_cells;
        expect(orc_step(&P, n, n_cells, n_inst, cell, inst, xi, v, 0, &st) == ORC_EINVAL, "bad cell accepted",
               case_id);
        cell[0] = keep;
    }
    free(members);
    free(perm);
    free(spec);
    free(count);
    free(cell);
    free(inst);
    free(xi);
    free(v);
    free(zeta);
}

int main(void)
{
    int id = 0;
    for (int32_t kernel = 0; kernel < 3; ++kernel)
        for (int32_t precision = 0; precision < 2; ++precision) {
            run_case(id++, 1, 1, 4096, kernel, precision, 1e6, 0);
            run_case(id++, 37, 1, 300, kernel, precision, 1e3, 1);
            run_case(id++, 6, 2, 64, kernel, precision, 1e-9, 0); /* p far above 1 */
            run_case(id++, 1, 1, 0, kernel, precision, 1e3, 0);   /* no SDs inside */
        }
    /* pair-level functions at their edges */
    orc_params P = {1, 0, 1500.0, 1.0, 1e3, 1.19e8, 8e3, 201.0, 40e-6, 600e-6, 3};
    expect(orc_gamma(1e300, 0.0, (int64_t)1 << 62, 1) == (int64_t)1 << 62, "gamma cap", id);
    expect(orc_gamma(0.0, 0.5, 5, 3) == 0, "gamma zero", id);
    expect(orc_cbrt(27.0) == 3.0 && orc_cbrtf(8.0f) == 2.0f, "cube root", id);
    expect(orc_kernel(&P, 1e-15, 1e-15) == 0.0, "K(r, r)", id);
    int64_t a = 4, b = 4;
    double va = 1.0, vb = 2.0;
    orc_update(1, &a, &b, &va, &vb);
    expect(a == 2 && b == 2 && va == 3.0 && vb == 3.0, "split", id);
    expect(orc_scale(&P, 2) > 0.0, "scale", id);
    if (failures) {
        fprintf(stderr, "%d failures\n", failures);
        return 1;
    }
    printf("oracle sanitized run: %d cases ok\n", id);
    return 0;
}
