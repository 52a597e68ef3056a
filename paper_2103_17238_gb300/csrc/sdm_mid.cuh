// Mid-size cells: above the shared-memory threshold of the block kernel
// (4096 SDs) and up to 65536 stored SDs.  One thread-block cluster of K CTAs
// per cell (K = 1, 2 or 4: up to 16384 SDs per CTA), persistent over a list
// of cells, every phase of the step in shared memory and distributed shared
// memory (DSMEM): no pass over global scratch, one launch per step and K.
//
// The permutation is the definition's sort of the live SDs by (key, rank).
// An entry is the key's top 48 bits above the 16-bit rank, so entries order
// as (key, rank) except between keys that share their top 48 bits (one pair
// in ~1e5 cells of 65536 SDs), which the in-bucket sort orders by their full
// keys, drawn again.  Per cell:
//   A  keys of the CTA's ranks (Philox, two per block), liveness, counts per
//      bucket (K x 2048 buckets on the keys' top bits, ~8 entries each);
//   B  bucket totals over the cluster (DSMEM reads), their scan, each
//      bucket's start position and each source CTA's offset in it;
//   C  keys drawn again and every entry stored at its position, in the CTA
//      that holds its bucket (the one whose range of positions, `chunk`
//      each, holds the bucket's start; DSMEM stores);
//   D  each CTA sorts the buckets it holds (one thread per bucket);
//   E  pairs (2l, 2l + 1): `chunk` is even, so a pair never straddles two
//      CTAs' ranges (its entries may, when a bucket does: DSMEM reads); the
//      pre-filter, the certified filter and the exact evaluation as in the
//      warp kernel, updates to global memory.
// Cluster barriers separate the phases; every CTA of a cluster runs the same
// cells and the same barriers, so no CTA waits on one that has left.
#pragma once

#include <cooperative_groups.h>

namespace sdm {

constexpr int kMidNT = 1024;
static_assert(kMidNT % 32 == 0 && kMidNT <= 1024 && ((4 << 11) / 4) % kMidNT == 0, "mid kernel: block shape");
constexpr int kMidSdPerCta = 16384; // stored SDs per CTA at most
constexpr int kMidMaxSd = 4 * kMidSdPerCta;
constexpr int kMidLBCta = 11;       // 2048 buckets per CTA
constexpr int kMidBucketMax = 2048; // entries a CTA holds beyond its range (one bucket's overhang)
constexpr int kMidCap = kMidSdPerCta + kMidBucketMax;

template <int K>
struct MidSmem {
    static constexpr int NB = K << kMidLBCta; // buckets of the cell
    static constexpr size_t off_E = 0;
    static constexpr size_t off_H = off_E + sizeof(uint64_t) * kMidCap;
    static constexpr size_t off_S = off_H + sizeof(uint32_t) * NB;
    static constexpr size_t off_L = off_S + sizeof(uint32_t) * (NB + 1);
    static constexpr size_t off_M = off_L + sizeof(uint32_t) * (kMidSdPerCta / 32);
    static constexpr size_t bytes = off_M + sizeof(uint32_t) * 16;
};

__device__ __forceinline__ uint64_t mid_key(uint64_t seed, uint32_t cell, int64_t s, uint32_t r)
{
    const uint4 w = draw4(seed, r >> 1, cell, s, 0u);
    return (r & 1u) ? (((uint64_t)w.z << 32) | w.w) : (((uint64_t)w.x << 32) | w.y);
}

// the full-key order of two entries with equal 48-bit prefixes (rare)
__device__ __noinline__ bool mid_less_full(uint64_t a, uint64_t b, uint64_t seed, uint32_t cell, int64_t s)
{
    const uint32_t ra = (uint32_t)(a & 0xFFFFu), rb = (uint32_t)(b & 0xFFFFu);
    return key_less(mid_key(seed, cell, s, ra), ra, mid_key(seed, cell, s, rb), rb);
}

// (key, rank) order of two entries; equal 48-bit prefixes take the full keys
__device__ __forceinline__ bool mid_less(uint64_t a, uint64_t b, uint64_t seed, uint32_t cell, int64_t s)
{
    if ((a >> 16) != (b >> 16))
        return a < b;
    return mid_less_full(a, b, seed, cell, s);
}

template <int K>
__global__ void __launch_bounds__(kMidNT, 1) mid_cell_kernel(const WorkItem *__restrict__ items, int32_t n_items,
                                                            InstDev *const *__restrict__ insts, int64_t step_offset)
{
    namespace cg = cooperative_groups;
    constexpr int NB = MidSmem<K>::NB;
    constexpr int LBT = kMidLBCta + (K == 1 ? 0 : (K == 2 ? 1 : 2)); // log2 NB
    constexpr unsigned FULL = 0xFFFFFFFFu;
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned me = cluster.block_rank();
    extern __shared__ __align__(16) unsigned char mid_smem[];
    uint64_t *E = reinterpret_cast<uint64_t *>(mid_smem + MidSmem<K>::off_E);
    uint32_t *H = reinterpret_cast<uint32_t *>(mid_smem + MidSmem<K>::off_H);
    uint32_t *S = reinterpret_cast<uint32_t *>(mid_smem + MidSmem<K>::off_S);
    uint32_t *Lm = reinterpret_cast<uint32_t *>(mid_smem + MidSmem<K>::off_L);
    uint32_t *M = reinterpret_cast<uint32_t *>(mid_smem + MidSmem<K>::off_M);
    // M[0 .. K): CTA totals of the bucket chunks; M[8]: a bucket too large
    // (any CTA); M[9 .. 9 + K]: first position held by each CTA, then n_c
    // another CTA's arrays through the cluster's shared-memory window (one
    // address translation, computed where it is used)
    auto Er = [&](unsigned c) { return cluster.map_shared_rank(E, c); };
    auto Hr = [&](unsigned c) { return cluster.map_shared_rank(H, c); };
    auto Sr = [&](unsigned c) { return cluster.map_shared_rank(S, c); };
    auto Mr = [&](unsigned c) { return cluster.map_shared_rank(M, c); };
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    __shared__ uint32_t s_warp[32];
    auto csync = [&]() { // a block barrier for one CTA, the cluster's otherwise
        if constexpr (K == 1)
            __syncthreads();
        else
            cluster.sync();
    };
    const int n_clusters = gridDim.x / K;
    const int cid = blockIdx.x / K;
    // cells come sorted by size, largest first, and are dealt in a snake
    // order (round r: cluster i takes cell r C + i, or r C + C - 1 - i for odd
    // r), which evens out the clusters' total work
    for (int round = 0;; ++round) {
        const int it = round * n_clusters + ((round & 1) ? n_clusters - 1 - cid : cid);
        if (it >= n_items)
            break;
        const WorkItem W = items[it];
        InstDev *__restrict__ P = insts[W.inst];
        const int64_t s = P->step + step_offset;
        const uint64_t seed = P->seed;
        const uint32_t cell = (uint32_t)W.cell;
        const int64_t *__restrict__ gxi = P->xi + W.off;
        double *__restrict__ gv = P->v + W.off;
        int64_t *__restrict__ gxw = P->xi + W.off;
        const int n = W.n;                                // stored SDs (even)
        const int m = ((n + K - 1) / K + 1) & ~1;          // ranks per CTA (even)
        const int r0 = (int)me * m, r1 = min(n, r0 + m);  // this CTA's ranks

        // ---- A: counts per bucket of this CTA's live SDs
        for (int b = t; b < NB; b += kMidNT)
            H[b] = 0;
        for (int w = t; w < kMidSdPerCta / 32; w += kMidNT)
            Lm[w] = 0;
        if (t == 0)
            M[8] = 0;
        __syncthreads();
        // warp-uniform trip count (the liveness bits are gathered by ballots:
        // a warp covers 64 consecutive ranks, two words of the mask)
        for (int q0 = (r0 >> 1) + (t & ~31); 2 * q0 < r1; q0 += kMidNT) {
            const int q = q0 + lane;
            const bool in = 2 * q < r1;
            uint4 w = make_uint4(0u, 0u, 0u, 0u);
            longlong2 x2 = make_longlong2(0, 0);
            if (in) {
                w = draw4(seed, (uint32_t)q, cell, s, 0u);
                x2 = reinterpret_cast<const longlong2 *>(gxi)[q];
                if ((q & 3) == 0) // bring the volumes into L2 for the pair phase
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(gv + 2 * q));
            }
            if (x2.x > 0)
                atomicAdd(&H[w.x >> (32 - LBT)], 1u);
            if (x2.y > 0)
                atomicAdd(&H[w.z >> (32 - LBT)], 1u);
            // bit 2 lane + h of the warp's 64 ranks: even ranks from one ballot,
            // odd ones from the other, interleaved into the two words
            const unsigned ev = __ballot_sync(FULL, x2.x > 0), od = __ballot_sync(FULL, x2.y > 0);
            if (lane < 2) {
                uint32_t word = 0;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int src = 16 * lane + k;
                    word |= ((ev >> src) & 1u) << (2 * k);
                    word |= ((od >> src) & 1u) << (2 * k + 1);
                }
                const int i0 = 2 * q0 - r0; // even, a multiple of 64 within the CTA's ranks
                if (i0 + 32 * lane < m)
                    Lm[(i0 >> 5) + lane] = word;
            }
        }
        csync(); // [1] every CTA's counts are in place

        // ---- B: totals of this CTA's chunk of buckets, their scan, starts
        constexpr int BPT = (NB / K) / kMidNT; // buckets per thread in the chunk (2)
        const int b0 = (int)me * (NB / K) + t * BPT;
        uint32_t cnt[BPT][K], tot[BPT], run = 0;
#pragma unroll
        for (int j = 0; j < BPT; ++j) {
            tot[j] = 0;
#pragma unroll
            for (int c = 0; c < K; ++c) {
                cnt[j][c] = Hr(c)[b0 + j];
                tot[j] += cnt[j][c];
            }
            run += tot[j];
            if (tot[j] > (uint32_t)kMidBucketMax)
                M[8] = 1;
        }
        // block exclusive scan of the per-thread sums
        uint32_t incl = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, d);
            if (lane >= d)
                incl += y;
        }
        if (lane == 31)
            s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t v = lane < kMidNT / 32 ? s_warp[lane] : 0u, vi = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, vi, d);
                if (lane >= d)
                    vi += y;
            }
            s_warp[lane] = vi - v;
            if (lane == 31) { // this chunk's total to every CTA
#pragma unroll
                for (int c = 0; c < K; ++c)
                    Mr(c)[me] = vi;
            }
        }
        __syncthreads();
        const uint32_t excl_local = s_warp[warp] + incl - run;
        const uint32_t bad_local = M[8];
        csync(); // [2] chunk totals everywhere
        uint32_t base = 0, n_c = 0;
#pragma unroll
        for (int c = 0; c < K; ++c) {
            base += c < (int)me ? M[c] : 0u;
            n_c += M[c];
        }
        {
            uint32_t p = base + excl_local;
#pragma unroll
            for (int j = 0; j < BPT; ++j) {
                // start of the bucket everywhere; each source's offset in it to the source
                uint32_t o = p;
#pragma unroll
                for (int c = 0; c < K; ++c) {
                    Sr(c)[b0 + j] = p;
                    Hr(c)[b0 + j] = o;
                    o += cnt[j][c];
                }
                p += tot[j];
            }
        }
        if (bad_local && t == 0) {
#pragma unroll
            for (int c = 0; c < K; ++c)
                atomicOr(&Mr(c)[8], 1u);
        }
        if (me == 0 && t == 0) {
#pragma unroll
            for (int c = 0; c < K; ++c)
                Sr(c)[NB] = n_c;
        }
        csync(); // [3] starts, offsets and the overflow flag everywhere
        // positions are dealt to the CTAs in ranges of `chunk` (even); a
        // bucket is held by the CTA whose range holds its start
        const uint32_t chunk = ((n_c + K - 1) / K + 1) & ~1u;
        auto holder = [&](uint32_t b) -> uint32_t { // min(K - 1, S[b] / chunk) by comparisons
            uint32_t h = 0;
            const uint32_t sb = S[b];
#pragma unroll
            for (int c = 1; c < K; ++c)
                h += sb >= (uint32_t)c * chunk ? 1u : 0u;
            return h;
        };
        const bool skip = M[8] != 0 || n_c < 2; // uniform over the cluster
        if (M[8] != 0 && me == 0 && t == 0)
            atomicOr(&P->status, 2u); // a bucket beyond the CTA's room: the cell is left as it was
        if (!skip) {
            // ---- C: entries to their positions
            for (int q = (r0 >> 1) + t; 2 * q < r1; q += kMidNT) {
                const int i = 2 * q - r0;
                const uint32_t lw = Lm[i >> 5] >> (i & 31);
                if ((lw & 3u) == 0)
                    continue;
                const uint4 w = draw4(seed, (uint32_t)q, cell, s, 0u);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!((lw >> h) & 1u))
                        continue;
                    const uint64_t key = h ? (((uint64_t)w.z << 32) | w.w) : (((uint64_t)w.x << 32) | w.y);
                    const uint32_t r = (uint32_t)(2 * q + h);
                    const uint64_t e = (key & ~0xFFFFull) | r;
                    const uint32_t b = (uint32_t)(key >> (64 - LBT));
                    const uint32_t pos = atomicAdd(&H[b], 1u);
                    const uint32_t hd = holder(b);
                    Er(hd)[pos - hd * chunk] = e;
                }
            }
        }
        csync(); // [4] every entry in place
        if (!skip) {
            // ---- D: sort the buckets this CTA holds
            // buckets held: [first b with holder >= me, first b with holder >= me + 1)
            auto first_held = [&](uint32_t h) -> uint32_t { // first bucket whose start is >= h chunk
                uint32_t lo = 0, hi = NB;
                const uint32_t lim = h * chunk;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (S[mid] < lim)
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                return lo;
            };
            const uint32_t bl = me == 0 ? 0u : first_held(me);
            const uint32_t bh = me == (unsigned)K - 1 ? (uint32_t)NB : first_held(me + 1);
            const uint32_t own0 = me * chunk;
            for (uint32_t b = bl + t; b < bh; b += kMidNT) {
                uint64_t *a = E + (S[b] - own0);
                const int k = (int)(S[b + 1] - S[b]);
                for (int x = 1; x < k; ++x) { // insertion sort (about 8 entries)
                    const uint64_t v = a[x];
                    int y = x - 1;
                    while (y >= 0 && mid_less(v, a[y], seed, cell, s)) {
                        a[y + 1] = a[y];
                        --y;
                    }
                    a[y + 1] = v;
                }
            }
            if (t == 0)
                M[9] = me == 0 ? 0u : S[bl]; // first position this CTA holds
        }
        csync(); // [5] buckets sorted everywhere
        if (!skip) {
            // ---- E: pairs whose first position is in this CTA's range
            const uint32_t own0 = me * chunk;
            const uint32_t p_lo = min(n_c, own0), p_hi = min(n_c, own0 + chunk);
            const uint32_t first_mine = M[9];
            auto entry = [&](uint32_t p) -> uint32_t { // rank at position p
                if (p >= first_mine)
                    return (uint32_t)(E[p - own0] & 0xFFFFu);
                // held by an earlier CTA: the one holding the bucket that holds p
                // (the last bucket starting at or before p)
                uint32_t lo = 0, hi = NB;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (S[mid] <= p)
                        lo = mid;
                    else
                        hi = mid;
                }
                const uint32_t hd = holder(lo);
                return (uint32_t)(Er(hd)[p - hd * chunk] & 0xFFFFu);
            };
            const uint32_t n_pairs = n_c / 2;
            const float ratio_f = u32_to_f32_rn((n_c & 1u) ? n_c : n_c - 1u);
            const PairConsts C = pair_consts(P);
            const float sc = C.dtdvf * ratio_f;
            const uint32_t l_lo = p_lo / 2, l_hi = min(n_pairs, (p_hi + 1) / 2);
            for (uint32_t q = (l_lo >> 1) + t; 2 * q < l_hi; q += kMidNT) {
                // both pairs' ranks, then every multiplicity and volume they
                // need, in one round of loads that overlaps the Philox block
                uint32_t ra[2], rb[2];
                int64_t x0[2], x1[2];
                double v0[2], v1[2];
                bool in[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t l = 2 * q + h;
                    in[h] = l >= l_lo && l < l_hi;
                    ra[h] = in[h] ? entry(2 * l) : 0u;
                    rb[h] = in[h] ? entry(2 * l + 1) : 0u;
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    x0[h] = in[h] ? gxi[ra[h]] : 0;
                    x1[h] = in[h] ? gxi[rb[h]] : 0;
                    v0[h] = in[h] ? gv[ra[h]] : 1.0;
                    v1[h] = in[h] ? gv[rb[h]] : 1.0;
                }
                const uint4 w = draw4(seed, q, cell, s, 1u);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!in[h])
                        continue;
                    uint32_t a = ra[h], b = rb[h];
                    const uint32_t wa = h ? w.z : w.x, wb = h ? w.w : w.y;
                    int64_t xa = x0[h], xb = x1[h];
                    double va = v0[h], vb = v1[h];
                    if (xa < xb) { // j holds the larger multiplicity; ties keep the earlier
                        const uint32_t tr = a;
                        a = b;
                        b = tr;
                        const int64_t tx = xa;
                        xa = xb;
                        xb = tx;
                        const double tv = va;
                        va = vb;
                        vb = tv;
                    }
                    const uint32_t ha = (uint32_t)__double2hiint(va), hb = (uint32_t)__double2hiint(vb);
                    if (pair_prefilter_zero(C, sc, xa, ha, hb, wa))
                        continue;
                    const int32_t gf = pair_gamma_filter(C, ratio_f, xa, ha, hb, wa);
                    int64_t g = 0;
                    if (gf > 0)
                        g = cap_gamma(gf, xa, xb);
                    else if (gf < 0)
                        g = pair_gamma_exact(P, n_c, xa, xb, va, vb, wa, wb);
                    if (g > 0) {
                        const bool split = shima_update(g, xa, xb, va, vb);
                        gxw[a] = xa;
                        gxw[b] = xb;
                        gv[b] = vb;
                        if (split)
                            gv[a] = va;
                    }
                }
            }
        }
        csync(); // [6] the cell's shared memory is free again
    }
}

} // namespace sdm
