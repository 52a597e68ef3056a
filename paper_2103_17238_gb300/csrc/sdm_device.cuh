// Device arithmetic of one SDM coalescence step: Philox4x32-10 streams, the
// cube root, Rogers-Yau terminal velocity, collision kernels, the collision
// count gamma and the Shima update.
//
// GB300 note.  Blackwell Ultra runs binary64 at a small fraction of its
// binary32 rate, yet the step must reproduce a binary64 definition bit for
// bit.  Each pair therefore first evaluates p in binary32 together with a
// rigorous bound on its distance from the binary64 value; when
// p + bound < u the pair certainly has gamma = 0 (the common case: p is a
// few percent) and nothing else is computed.  Only pairs that may collide
// run the exact binary64 evaluation, with explicit round-to-nearest
// intrinsics so that no multiply-add is contracted.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sdm {

enum : int32_t { KERNEL_GOLOVIN = 0, KERNEL_GEOMETRIC = 1, KERNEL_LONG = 2 };
enum : int32_t { PREC_FP64 = 0, PREC_KFP32 = 1 };

// Per-run parameters, one record per context in device memory.
struct InstDev {
    int64_t *xi;             // multiplicities, storage order
    double *v;               // volumes, storage order
    const int32_t *cell_off; // n_cells + 1 storage offsets (every cell starts at an even slot)
    uint64_t seed;
    int64_t step;            // index of the next step
    double dtdv;             // dt / dv
    double b;                // Golovin constant
    double k1, k2, k3, r1, r2;
    float bf, k1f, k2f, k3f, r1f, r2f; // binary32 roundings of the above
    float dtdvf;                       // dt / dv rounded to binary32 (filter only)
    float pre_c[3];  // pre-filter: p <= pre_c[regime] f(v_max) xi_j scale (rounded up; pair_prefilter_zero)
    float pre_v[2];  // pre-filter: volumes of the regime bounds r1, r2 (rounded down)
    int32_t kernel, precision, n_cells;
    uint32_t status; // bit 0: a bounded device wait gave up (reported as SDM_ETIMEOUT)
};

struct __align__(16) WorkItem {
    int32_t inst; // index into the batch's table of InstDev pointers
    int32_t cell; // the cell's index in the random streams (its run's cell_base + cell)
    int32_t off;  // the cell's first storage slot (the plan is rebuilt when the layout changes)
    int32_t n;    // the cell's storage slots
};

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
// products with the Weyl key schedule.
__device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

__device__ __forceinline__ uint32_t mullo32(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("mul.lo.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// Separate high and low 32-bit products issue fewer instructions here than
// one 64-bit product (measured on sm_103a).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t h0 = mulhi32(0xD2511F53u, c.x), l0 = mullo32(0xD2511F53u, c.x);
        const uint32_t h1 = mulhi32(0xCD9E8D57u, c.z), l1 = mullo32(0xCD9E8D57u, c.z);
        c = make_uint4(h1 ^ c.y ^ k.x, l1, h0 ^ c.w ^ k.y, l0);
    }
    return c;
}

// Stream layout: ctr = (index >> 1, cell, s_lo, s_hi31 | tag << 31),
// key = seed.  Tag 0: sort keys by SD rank; tag 1: pair uniforms by pair.
__device__ __forceinline__ uint4 draw4(uint64_t seed, uint32_t half_index, uint32_t cell, int64_t s,
                                       uint32_t tag)
{
    const uint4 c = make_uint4(half_index, cell, (uint32_t)((uint64_t)s),
                               ((uint32_t)((uint64_t)s >> 32) & 0x7FFFFFFFu) | (tag << 31));
    return philox4x32_10(c, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// 53-bit uniform m * 2^-53 from the word pair (wa, wb).
__device__ __forceinline__ double uniform53(uint32_t wa, uint32_t wb)
{
    const uint64_t m = ((uint64_t)wa << 21) | (uint64_t)(wb >> 11);
    return __dmul_rn(__ull2double_rn(m), 0x1p-53);
}

// A binary32 lower bound of the same uniform: its top 23 bits, exactly
// ((wa >> 9) 2^-23 built as a float in [1, 2) minus 1).
__device__ __forceinline__ float uniform_lo23(uint32_t wa) { return __uint_as_float(0x3F800000u | (wa >> 9)) - 1.0f; }

// ------------------------------------------------------------ conversions
// Blackwell Ultra issues F2F.F64 and I2F.S64 on its narrow binary64 pipe, so
// the common path converts with integer operations instead.  Both are
// exactly round-to-nearest-even, like (float)x in C.

// x in the normal binary32 range (in_range reports it); sign kept.
__device__ __forceinline__ float d2f_rn(double x, bool &in_range)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t e = (hi >> 20) & 0x7FFu;
    in_range = (e - 897u) < 253u; // binary32 exponent field 1 .. 253 before rounding
    const uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const uint32_t rest = lo & 0x1FFFFFFFu;
    uint32_t bits = ((e - 896u) << 23) + m;
    bits += (uint32_t)(rest > 0x10000000u) | ((uint32_t)(rest == 0x10000000u) & (m & 1u));
    return __uint_as_float(bits | (hi & 0x80000000u));
}

// two exact 16-bit halves, one rounding in the final fused add
__device__ __forceinline__ float u32_to_f32_rn(uint32_t u)
{
    const float lo = __uint_as_float((u & 0xFFFFu) | 0x4B000000u) - 8388608.0f;
    const float hi = __uint_as_float((u >> 16) | 0x4B000000u) - 8388608.0f;
    return __fmaf_rn(hi, 65536.0f, lo);
}

__device__ __forceinline__ float xi_to_f32_rn(int64_t x)
{
    return ((uint64_t)x >> 32) == 0 ? u32_to_f32_rn((uint32_t)x) : __ll2float_rn(x);
}

// ------------------------------------------------------------- cube root
// The library's cube root is a fixed sequence of IEEE operations so that its
// result is reproducible: x = f 2^E (f in [1,2)), E = 3k + j, m = f 2^j in
// [1,8); a quadratic seed for f^(-1/3) scaled by 2^(-j/3), two binary32
// Newton steps for m^(-1/3) (z += z (1 - m z^3) / 3); then y = m z^2 and
// R = z^2 / 3, two binary64 steps y -= (y^3 - m) R, and y 2^k.
// Binary64 result within 1 ulp; binary32 twin within 1 ulp.
constexpr float kCbrtP0 = 0x1.610e12p+0f;
constexpr float kCbrtP1 = -0x1.e43e5cp-2f;
constexpr float kCbrtP2 = 0x1.72f4a4p-4f;
constexpr float kThirdF = 0x1.555556p-2f;
constexpr double kPi = 0x1.921fb54442d18p+1;      // pi rounded to binary64
constexpr double kVolToR3 = 0x1.e8ec8a4aeacc4p-3; // 0.75 / pi in binary64
constexpr float kPiF = 0x1.921fb6p+1f;            // the binary64 pi rounded to binary32
constexpr float kVolToR3F = 0x1.e8ec8ap-3f;       // 0.75 / pi rounded to binary32

__device__ __forceinline__ float inv_cbrt_seed(float ff, float mf, int j)
{
    const float cj = (j == 0) ? 1.0f : ((j == 1) ? 0x1.965feap-1f : 0x1.428a30p-1f);
    float z = __fmul_rn(kCbrtP2, ff);
    z = __fadd_rn(kCbrtP1, z);
    z = __fmul_rn(ff, z);
    z = __fadd_rn(kCbrtP0, z);
    z = __fmul_rn(z, cj);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        float t = __fmul_rn(z, z);
        t = __fmul_rn(t, z);
        t = __fmul_rn(mf, t);
        t = __fsub_rn(1.0f, t);
        t = __fmul_rn(t, z);
        t = __fmul_rn(t, kThirdF);
        z = __fadd_rn(z, t);
    }
    return z;
}

// x: positive normal binary64.
__device__ __forceinline__ double cbrt_exact(double x)
{
    const uint64_t bits = (uint64_t)__double_as_longlong(x);
    const int E = (int)((bits >> 52) & 0x7FF) - 1023;
    const int k = (E + 3069) / 3 - 1023;
    const int j = E - 3 * k;
    const uint64_t mant = bits & 0x000FFFFFFFFFFFFFull;
    const double f = __longlong_as_double((long long)(mant | (1023ull << 52)));
    const double m = __longlong_as_double((long long)(mant | ((uint64_t)(1023 + j) << 52)));
    const float ff = __double2float_rn(f);
    const float mf = __double2float_rn(m);
    const float z = inv_cbrt_seed(ff, mf, j);
    const float zz = __fmul_rn(z, z);
    double y = (double)__fmul_rn(mf, zz);
    const double R = (double)__fmul_rn(zz, kThirdF);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        double c = __dmul_rn(y, y);
        c = __dmul_rn(c, y);
        c = __dsub_rn(c, m);
        c = __dmul_rn(c, R);
        y = __dsub_rn(y, c);
    }
    return __dmul_rn(y, __longlong_as_double((long long)((uint64_t)(k + 1023) << 52)));
}

// x: positive normal binary32.
__device__ __forceinline__ float cbrt32(float x)
{
    const uint32_t bits = __float_as_uint(x);
    const int E = (int)((bits >> 23) & 0xFF) - 127;
    const int k = (E + 381) / 3 - 127;
    const int j = E - 3 * k;
    const uint32_t mant = bits & 0x007FFFFFu;
    const float ff = __uint_as_float(mant | (127u << 23));
    const float mf = __uint_as_float(mant | ((uint32_t)(127 + j) << 23));
    const float z = inv_cbrt_seed(ff, mf, j);
    const float zz = __fmul_rn(z, z);
    float y = __fmul_rn(mf, zz);
    const float rf = __fmul_rn(zz, kThirdF);
    float c = __fmul_rn(y, y);
    c = __fmul_rn(c, y);
    c = __fsub_rn(c, mf);
    c = __fmul_rn(c, rf);
    y = __fsub_rn(y, c);
    return __fmul_rn(y, __uint_as_float((uint32_t)(k + 127) << 23));
}

__device__ __forceinline__ double radius_exact(double v) { return cbrt_exact(__dmul_rn(v, kVolToR3)); }
__device__ __forceinline__ float radius32(float v) { return cbrt32(__fmul_rn(v, kVolToR3F)); }

// ------------------------------------------------------ terminal velocity
__device__ __forceinline__ double vt_exact(const InstDev &P, double r)
{
    if (r < P.r1)
        return __dmul_rn(P.k1, __dmul_rn(r, r));
    if (r < P.r2)
        return __dmul_rn(P.k2, r);
    return __dmul_rn(P.k3, __dsqrt_rn(r));
}

// ------------------------------------------------ Long's collision efficiency
// Long (1974): with R the larger and r the smaller radius of the pair,
// E = max(c1 R^2 (1 - c2 / r), E_min) for R <= R_lim and 1 above, with
// c1 = 4.5e8 m^-2, c2 = 3e-6 m, E_min = 1e-3, R_lim = 50 um (the cgs
// constants 4.5e4 cm^-2 and 3e-4 cm in SI).  The kernel is the geometric
// sweep-out times E.  Both precisions use the binary64 constants' values
// (binary32: their roundings), in this operation order.
constexpr double kLongC1 = 4.5e8, kLongC2 = 3e-6, kLongEmin = 1e-3, kLongRlim = 50e-6;
constexpr float kLongC1F = (float)kLongC1, kLongC2F = (float)kLongC2, kLongEminF = (float)kLongEmin,
                kLongRlimF = (float)kLongRlim;

__device__ __forceinline__ double efficiency_long_exact(double rj, double rk)
{
    const double R = rj > rk ? rj : rk, r = rj > rk ? rk : rj;
    if (R > kLongRlim)
        return 1.0;
    const double e = __dmul_rn(__dmul_rn(kLongC1, __dmul_rn(R, R)), __dsub_rn(1.0, __ddiv_rn(kLongC2, r)));
    return e < kLongEmin ? kLongEmin : e;
}

__device__ __forceinline__ float efficiency_long32(float rj, float rk)
{
    const float R = rj > rk ? rj : rk, r = rj > rk ? rk : rj;
    if (R > kLongRlimF)
        return 1.0f;
    const float e = __fmul_rn(__fmul_rn(kLongC1F, __fmul_rn(R, R)), __fsub_rn(1.0f, __fdiv_rn(kLongC2F, r)));
    return e < kLongEminF ? kLongEminF : e;
}

// --------------------------------------------------------------- p and gamma
// Exact binary64 probability (the definition).
__device__ __noinline__ double probability_exact(const InstDev &P, double scale, int64_t xi_j, double vj,
                                                 double vk)
{
    double K;
    if (P.kernel == KERNEL_GOLOVIN) {
        K = __dmul_rn(P.b, __dadd_rn(vj, vk));
    } else {
        const double rj = radius_exact(vj), rk = radius_exact(vk);
        const double s = __dadd_rn(rj, rk);
        K = __dmul_rn(__dmul_rn(kPi, __dmul_rn(s, s)), fabs(__dsub_rn(vt_exact(P, rj), vt_exact(P, rk))));
        if (P.kernel == KERNEL_LONG)
            K = __dmul_rn(K, efficiency_long_exact(rj, rk));
    }
    return __dmul_rn(__dmul_rn(K, __ll2double_rn(xi_j)), scale);
}

// gamma = min(ceil(p - u), floor(xi_j / xi_k)), the comparison made in
// binary64 before any integer conversion.
__device__ __forceinline__ int64_t gamma_exact(double p, double u, int64_t xi_j, int64_t xi_k)
{
    const double g = ceil(__dsub_rn(p, u));
    if (!(g >= 1.0))
        return 0;
    const int64_t q = xi_j / xi_k;
    if (g >= __ll2double_rn(q))
        return q;
    return __double2ll_rz(g);
}

// dt/dV [n_c (n_c - 1) / 2] / floor(n_c / 2), once per cell.  The ratio is
// exactly n_c - 1 for even n_c and n_c for odd n_c, so the IEEE quotient of
// the definition equals that integer and no division is needed.
__device__ __forceinline__ double cell_scale(double dtdv, int64_t n_c)
{
    const int64_t ratio = (n_c & 1) ? n_c : n_c - 1;
    return __dmul_rn(dtdv, __ll2double_rn(ratio));
}

// Per-run constants of the pair arithmetic, loaded once per cell.
struct PairConsts {
    float bf, k1f, k2f, k3f, r1f, r2f;
    float dtdvf;                  // dt / dV rounded to binary32 (filter only)
    float pre_c[3], pre_v[2];     // the pre-filter's constants
    float r1_lo, r1_hi, r2_lo, r2_hi; // regime bounds widened by 2^-14 (filter only)
    int32_t kernel, precision;
};

__device__ __forceinline__ PairConsts pair_consts(const InstDev *P)
{
    PairConsts c;
    c.bf = P->bf;
    c.k1f = P->k1f;
    c.k2f = P->k2f;
    c.k3f = P->k3f;
    c.r1f = P->r1f;
    c.r2f = P->r2f;
    c.dtdvf = P->dtdvf;
    c.pre_c[0] = P->pre_c[0];
    c.pre_c[1] = P->pre_c[1];
    c.pre_c[2] = P->pre_c[2];
    c.pre_v[0] = P->pre_v[0];
    c.pre_v[1] = P->pre_v[1];
    c.r1_lo = c.r1f * (1.0f - 0x1p-14f);
    c.r1_hi = c.r1f * (1.0f + 0x1p-14f);
    c.r2_lo = c.r2f * (1.0f - 0x1p-14f);
    c.r2_hi = c.r2f * (1.0f + 0x1p-14f);
    c.kernel = P->kernel;
    c.precision = P->precision;
    return c;
}

__device__ __forceinline__ float vt32c(const PairConsts &C, float r)
{
    if (r < C.r1f)
        return __fmul_rn(C.k1f, __fmul_rn(r, r));
    if (r < C.r2f)
        return __fmul_rn(C.k2f, r);
    return __fmul_rn(C.k3f, __fsqrt_rn(r));
}

// ------------------------------------------------------------- the filter
// Filter-grade helpers: each has a stated relative error e, and the filter's
// margin covers their sum with a wide factor.
//   hi2f           e < 2^-20 (the binary64's top 20 mantissa bits)
//   xi2f           e < 2^-23 (truncating conversion)
//   cbrt_filter    e < 2^-18.9 (lg2/ex2 approximations; maximum 2^-18.99
//                  measured exhaustively over every binary32 in
//                  [2^-110, 2^110) on sm_103a against the binary64 cube root)

__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float cbrt_filter(float x) { return ex2_approx(lg2_approx(x) * 0x1.555556p-2f); }


// Binary32 image of a positive binary64 from its high word alone: the top
// 20 mantissa bits (relative error < 2^-20), exponent rebiased.  in_range:
// the result is a normal binary32 (exponent field 1..253).
__device__ __forceinline__ float hi2f(uint32_t hi, bool &in_range)
{
    in_range = (hi - (897u << 20)) < (253u << 20);
    return __uint_as_float((hi << 3) - (896u << 23));
}

// Binary32 image of a multiplicity x >= 1 truncated to 24 bits (relative
// error < 2^-23), built on the integer pipe: 64-bit conversions would run on
// the scarce binary64 pipe.
__device__ __forceinline__ float xi2f(int64_t x)
{
    const uint64_t u = (uint64_t)x;
    const uint32_t lz = (uint32_t)__clzll((long long)u); // < 64 for x >= 1
    const uint32_t top = (uint32_t)((u << lz) >> 40);    // leading 24 bits, bit 23 set
    return __uint_as_float(((190u - lz) << 23) + (top & 0x7FFFFFu));
}

// The binary64 value of a multiplicity 0 <= x < 2^53 (exact) built on the
// integer pipe; larger x by the conversion instruction (round to nearest).
__device__ __forceinline__ double xi2d(int64_t x)
{
    const uint64_t u = (uint64_t)x;
    if (u >> 53)
        return __ll2double_rn(x);
    if (u == 0)
        return 0.0;
    const uint32_t lz = (uint32_t)__clzll((long long)u);           // 11 .. 63
    const uint64_t mant = (u << (lz - 11)) & 0x000FFFFFFFFFFFFFull; // 52 bits below the leading one
    return __longlong_as_double((long long)(((uint64_t)(1086u - lz) << 52) | mant));
}

// Fall speed for the filter; clears ok within 2^-14 of a regime boundary,
// where the filter's radius could fall on the other side of it.
__device__ __forceinline__ float vt_guarded(const PairConsts &C, float r, bool &ok)
{
    // regimes 1 and 2 by a select (no divergence); regime 3 (the largest
    // drops, rare) by a branch
    const bool reg1 = r < C.r1_lo;
    float t = reg1 ? C.k1f * (r * r) : C.k2f * r;
    ok &= reg1 | (r > C.r1_hi);
    if (r >= C.r2_lo) {
        ok &= r > C.r2_hi;
        t = C.k3f * sqrtf(r);
    }
    return t;
}

// The collision count ceil(p - u) of a pair (xi_j >= xi_k > 0) when the
// binary32 evaluation determines it, else -1 (before the cap at
// floor(xi_j / xi_k)).  vj_hi, vk_hi: high words of the binary64 volumes.
// With pf the filter's binary32 value of p and M a binary32 magnitude of all
// of p's terms (K evaluated with |v_t(r_j) - v_t(r_k)| replaced by the sum),
// the filter's error is below 2^-16.4 M (volumes 2^-20, radius 2^-18.8,
// squares and fall speeds 2^-17.7, the difference absolute in M) and the
// exact value's (binary64, or binary32 with a 1-ulp cube root) below
// 2^-19 M: together below 2^-16.1 M.  So with E = 2^-13 M + 2^-100 (over 8
// times that bound) and u in [u_lo, u_lo + 2^-23),
// p - u lies in [pf - E - u_hi, pf + E - u_lo], and the bounds, widened by
// the rounding of their own binary32 sums, pin ceil(p - u) when both fall in
// one interval (m - 1, m].  The filter abstains within 2^-14 of a
// terminal-velocity regime boundary (radius error 2^-18.8), when a binary32
// value leaves the normal range, and for counts above 2^16.
__device__ __forceinline__ int32_t pair_gamma_filter(const PairConsts &C, float ratio_f, int64_t xi_j,
                                                     uint32_t vj_hi, uint32_t vk_hi, uint32_t wa)
{
    const float u_lo = uniform_lo23(wa);
    bool ok, ok_k;
    const float vjf = hi2f(vj_hi, ok), vkf = hi2f(vk_hi, ok_k);
    ok &= ok_k;
    const float xjf = xi2f(xi_j);
    const float sc = C.dtdvf * ratio_f;
    float pf, mag;
    if (C.kernel == KERNEL_GOLOVIN) {
        const float K = C.bf * (vjf + vkf);
        pf = (K * xjf) * sc;
        mag = pf;
        ok &= K >= 0x1p-126f;
    } else {
        const float rj = cbrt_filter(vjf * kVolToR3F), rk = cbrt_filter(vkf * kVolToR3F);
        const float tj = vt_guarded(C, rj, ok), tk = vt_guarded(C, rk, ok);
        const float s = rj + rk;
        const float a = kPiF * (s * s);
        float K = a * fabsf(tj - tk);
        float km = a * (tj + tk);
        if (C.kernel == KERNEL_LONG) {
            // E and Em = c1 R^2 (1 + c2 / r) + E_min >= E: the error of the
            // filter's E is below 2^-16.9 Em (radii 2^-18.8, the quotient
            // 2^-21 with the approximate division, products), so K's bound
            // becomes (2^-16.4 + 2^-16.9) km Em < 2^-15.6 km Em, and E below
            // stays over 5 times the total.  Abstains within 2^-14 of R_lim.
            const float R = fmaxf(rj, rk), r = fminf(rj, rk);
            ok &= !(R > kLongRlimF * (1.0f - 0x1p-14f) && R < kLongRlimF * (1.0f + 0x1p-14f));
            if (R <= kLongRlimF) {
                const float c = kLongC1F * (R * R);
                const float q = __fdividef(kLongC2F, r);
                K *= fmaxf(c * (1.0f - q), kLongEminF);
                km *= c * (1.0f + q) + kLongEminF;
            }
        }
        pf = (K * xjf) * sc;
        mag = (km * xjf) * sc;
        ok &= km >= 0x1p-126f && (K == 0.0f || K >= 0x1p-126f);
    }
    const float E = mag * 0x1p-13f + 0x1p-100f;
    const float slack = (fabsf(pf) + E + 1.0f) * 0x1p-20f;
    const float hi = ((pf + E) - u_lo) + slack;
    if (ok && hi <= 0.0f)
        return 0;
    const float lo = ((pf - E) - (u_lo + 0x1p-23f)) - slack;
    const float m = ceilf(hi);
    if (!ok || ceilf(lo) != m || !(m <= 65536.0f))
        return -1;
    return (int32_t)m;
}

// A bound that settles most pairs before the filter: gamma = 0 is certain
// when p < u, and p <= B xi_j scale.  Golovin: K = b (v_j + v_k) <= 2 b v_max.
// Long: the geometric bound below times 1.125 >= Long's E (at most
// c1 R_lim^2), folded into pre_c on the host.
// Geometric: the fall speed never decreases with r (the Rogers-Yau regimes
// join with upward steps), so K = pi (r_j + r_k)^2 |v_t(r_j) - v_t(r_k)| <=
// 4 pi r_max^2 v_t(r_max), which in each regime is
//   r < r1:       4 pi k1 r^4    = C1 v^(4/3),  C1 = 4 pi k1 (3 / (4 pi))^(4/3)
//   r1 <= r < r2: 4 pi k2 r^3    = 3 k2 v
//   r >= r2:      4 pi k3 r^(5/2) = C3 v^(5/6), C3 = 4 pi k3 (3 / (4 pi))^(5/6).
// The regime is chosen from v_max (1 + 2^-10): near a bound the upper
// regime's formula, which is the larger one there (its speed jumps up),
// covers both sides.  pre_c (2 b, C1, 3 k2, C3) is rounded up and the regime
// volumes down on the host.  The binary32 evaluation underestimates B xi_j
// scale by less than 2^-15 (truncated v and xi, the scale's rounding, three
// products, lg2/ex2 approximations for the powers), and the exact p (binary64,
// or binary32 with the 1-ulp radius) exceeds the bound's real value by less
// than 2^-17: so bound (1 + 2^-8) < u_lo (u's exact lower bound) proves
// p < u.  Out-of-range or underflowing values abstain (return false).
__device__ __forceinline__ bool pair_prefilter_zero(const PairConsts &C, float sc, int64_t xi_j, uint32_t vj_hi,
                                                    uint32_t vk_hi, uint32_t wa)
{
    bool ok, ok_k;
    const float vjf = hi2f(vj_hi, ok), vkf = hi2f(vk_hi, ok_k);
    ok &= ok_k;
    const float vmax = fmaxf(vjf, vkf);
    float bound;
    if (C.kernel == KERNEL_GOLOVIN) {
        bound = C.pre_c[0] * vmax;
    } else {
        const float vup = vmax * (1.0f + 0x1p-10f);
        if (vup < C.pre_v[1] && !(vup < C.pre_v[0])) {
            bound = C.pre_c[1] * vmax;
        } else {
            const bool stokes = vup < C.pre_v[0];
            const float t = ex2_approx(lg2_approx(vmax) * (stokes ? 4.0f / 3.0f : 5.0f / 6.0f));
            ok &= t >= 0x1p-100f;
            bound = (stokes ? C.pre_c[0] : C.pre_c[2]) * t;
        }
    }
    bound = (bound * xi2f(xi_j)) * sc;
    return ok && bound * (1.0f + 0x1p-8f) < uniform_lo23(wa);
}

// The same from full binary64 volumes.
__device__ __forceinline__ int32_t pair_gamma_filter(const PairConsts &C, float ratio_f, int64_t xi_j, double vj,
                                                     double vk, uint32_t wa)
{
    return pair_gamma_filter(C, ratio_f, xi_j, (uint32_t)__double2hiint(vj), (uint32_t)__double2hiint(vk), wa);
}

// gamma capped at floor(xi_j / xi_k) for a certain count g >= 1 (the
// comparison of the definition, made exactly in integers: g is small).
__device__ __forceinline__ int64_t cap_gamma(int32_t g, int64_t xi_j, int64_t xi_k)
{
    if (g == 1)
        return 1; // xi_j >= xi_k
    // g xi_k <= xi_j (no overflow: the 128-bit product's high word is zero)
    // means floor(xi_j / xi_k) >= g; only the capped case divides
    const uint64_t lo = (uint64_t)g * (uint64_t)xi_k;
    const uint64_t hi = __umul64hi((uint64_t)g, (uint64_t)xi_k);
    if (hi == 0 && lo <= (uint64_t)xi_j)
        return g;
    return xi_j / xi_k;
}

// ------------------------------------------------------------ exact gamma
// The definition: p in binary64 (FP64 mode) or binary32 widened (KFP32
// mode), then gamma.  Called for the pairs the filter could not decide,
// compacted so that every lane of a warp has one.
__device__ __forceinline__ int64_t pair_gamma_exact(const InstDev *P, uint32_t n_c, int64_t xi_j, int64_t xi_k,
                                                    double vj, double vk, uint32_t wa, uint32_t wb)
{
    const double scale = cell_scale(P->dtdv, (int64_t)n_c);
    double p;
    if (P->precision == PREC_KFP32) {
        const PairConsts C = pair_consts(P);
        bool in_j, in_k;
        const float vjf = d2f_rn(vj, in_j), vkf = d2f_rn(vk, in_k);
        const float xjf = xi_to_f32_rn(xi_j);
        const float scale_f = __double2float_rn(scale);
        float K;
        if (C.kernel == KERNEL_GOLOVIN) {
            K = __fmul_rn(C.bf, __fadd_rn(vjf, vkf));
        } else {
            const float rj = radius32(vjf), rk = radius32(vkf);
            const float s = __fadd_rn(rj, rk);
            K = __fmul_rn(__fmul_rn(kPiF, __fmul_rn(s, s)), fabsf(__fsub_rn(vt32c(C, rj), vt32c(C, rk))));
            if (C.kernel == KERNEL_LONG)
                K = __fmul_rn(K, efficiency_long32(rj, rk));
        }
        p = (double)__fmul_rn(__fmul_rn(K, xjf), scale_f);
    } else {
        p = probability_exact(*P, scale, xi_j, vj, vk);
    }
    return gamma_exact(p, uniform53(wa, wb), xi_j, xi_k);
}

// Shima update for gamma > 0.  Returns true when the j SD's volume changed
// (the split case).
__device__ __forceinline__ bool shima_update(int64_t gamma, int64_t &xi_j, int64_t &xi_k, double &vj, double &vk)
{
    // (double)1 * v_j is v_j exactly: one binary64 add for the common gamma = 1
    double t = vj;
    if (gamma != 1)
        t = __dmul_rn(__ll2double_rn(gamma), vj);
    const double vnew = __dadd_rn(vk, t);
    const int64_t rem = xi_j - gamma * xi_k;
    if (rem > 0) {
        xi_j = rem;
        vk = vnew;
        return false;
    }
    const int64_t h = xi_k / 2;
    xi_j = h;
    xi_k = xi_k - h;
    vj = vnew;
    vk = vnew;
    return true;
}


} // namespace sdm
