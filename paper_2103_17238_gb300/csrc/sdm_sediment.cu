// Sedimentation step (sdm_set_positions, sdm_sedimentation_step,
// sdm_get_positions in include/sdm.h).
//
// The paper lists particle displacement among the dynamics of its framework
// and shows sedimenting drizzle in its 2-D example; it prints no formulae.
// Reading: every live SD falls by its Rogers-Yau speed times dt, the speed
// taken from the binary32 radius twin of its volume (the KFP32 arithmetic)
// and the distance widened exactly to binary64; positions are heights above
// the bottom of the SD's cell, so a step needs no division.
//
// One step on the device:
//   sed_move_kernel      per slot (four per thread): the fall, the new group
//                        of every SD (the cells, then n_cells for outside the
//                        domain) as a key in SD-id order, counts per new
//                        group, the water that leaves through the bottom;
//   sed_scan_kernel      new group offsets (unpadded and padded to even
//                        slots) and the precipitated total, in fixed order;
//   radix_*_kernel       stable LSD radix sort of the keys, 8-bit digits
//                        (SD-id order in, so equal groups keep increasing
//                        id): per-tile digit counts, a scan of each digit's
//                        row, a scan of the digit totals, a ranked scatter;
//   sed_gather_kernel    the new layout, gathered from the old one;
//   sed_pad_kernel       its padding slots.
// The scan, the padding, the refresh of the context's own launch plan and
// the read-back run on a side stream beside the radix sort.
// The two layouts swap; the host reads the new offsets for the launch plan.
//
// Compiled as part of the library's single translation unit (included at the
// end of sdm_runtime.cu).

namespace {

constexpr int kSedNT = 256;
constexpr int kRadixNT = 256;
constexpr int kRadixRounds = 16;
constexpr int kRadixTile = kRadixNT * kRadixRounds; // keys per block and pass
constexpr int kRadixBuckets = 256;                  // 8-bit digits

// ------------------------------------------------------------------ kernels
// zeta of every slot from z (SD-id order): z - (level) dz with level =
// (cbase + c) / nx, which must lie in [0, dz) (zeta_in: z already holds
// zeta); flags bit 0 and the first bad id on failure.  SDs outside the
// domain and padding slots get zeta 0.  group[slot] = the slot's group.
__global__ void __launch_bounds__(kSedNT) sed_set_kernel(const int32_t *__restrict__ cell_off, int32_t n_cells,
                                                         int64_t n_slots, const int32_t *__restrict__ id_of_slot,
                                                         const double *__restrict__ z, int32_t nx, double dz,
                                                         int32_t cbase, int zeta_in,
                                                         double *__restrict__ zeta, int32_t *__restrict__ group,
                                                         uint32_t *__restrict__ flags,
                                                         unsigned long long *__restrict__ bad)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int g = gw; g <= n_cells; g += nw) {
        const int64_t lo = cell_off[g], hi = g < n_cells ? cell_off[g + 1] : n_slots;
        const double base = zeta_in ? 0.0 : __dmul_rn((double)((g + cbase) / nx), dz);
        for (int64_t s = lo + lane; s < hi; s += 32) {
            const int32_t id = id_of_slot[s];
            double zt = 0.0;
            if (id >= 0 && g < n_cells) {
                // + 0 turns a -0 height into +0 (the fall tests signs bitwise)
                zt = __dadd_rn(__dsub_rn(z[id], base), 0.0);
                if (!(zt >= 0.0 && zt < dz)) {
                    atomicOr(flags, 1u);
                    atomicMin(bad, (unsigned long long)id);
                    zt = 0.0;
                }
            }
            zeta[s] = zt;
            group[s] = g;
        }
    }
}

// z[id] = ((cbase + c) / nx) dz + zeta (0 outside) and cell[id] = c (-1
// outside).  zeta_out[id] = zeta of the slot, and gcell[id] = cbase + c
// inside, else emig[id]: the cell of another piece of the grid that the SD
// entered through this piece's bottom in the last sedimentation step, or -1
// (zeta_out then its height in that cell, else 0).
__global__ void __launch_bounds__(kSedNT) sed_get_kernel(const int32_t *__restrict__ cell_off, int32_t n_cells,
                                                         int64_t n_slots, const int32_t *__restrict__ id_of_slot,
                                                         const double *__restrict__ zeta, int32_t nx, double dz,
                                                         int32_t cbase, const int32_t *__restrict__ emig,
                                                         double *__restrict__ z, int32_t *__restrict__ cell,
                                                         double *__restrict__ zeta_out, int32_t *__restrict__ gcell)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int g = gw; g <= n_cells; g += nw) {
        const int64_t lo = cell_off[g], hi = g < n_cells ? cell_off[g + 1] : n_slots;
        const double base = g < n_cells && z ? __dmul_rn((double)((g + cbase) / nx), dz) : 0.0;
        for (int64_t s = lo + lane; s < hi; s += 32) {
            const int32_t id = id_of_slot[s];
            if (id < 0)
                continue;
            if (z)
                z[id] = g < n_cells ? __dadd_rn(base, zeta[s]) : 0.0;
            if (cell)
                cell[id] = g < n_cells ? g : -1;
            if (zeta_out)
                zeta_out[id] = zeta[s];
            if (gcell)
                gcell[id] = g < n_cells ? g + cbase : (emig ? emig[id] : -1);
        }
    }
}

// The fall of every SD, four slots per thread (grid-stride, all loads
// issued before use).  key[id] = its new group (n_cells: outside), val[id]
// = its slot, zeta_new[slot] = its new height; counts[new group] (one
// atomic per run of equal groups among a warp's 32 consecutive slots);
// precip_part[block] = sum of xi v of the SDs that fell through the bottom
// of the grid (thread order fixed, then a fixed tree over the block).
// Levels are counted from the grid's bottom (cell cbase + c): an SD that
// leaves this piece's lowest level into a level of another piece becomes
// outside here, with emig[id] = its new cell there and zeta_new its height
// in it (emig[id] = -1 for every other SD).
constexpr int kSedU = 4;
constexpr int kSedMaxBlocks = 4096;

// The binary64 value of a binary32, exactly, on the integer pipe for normal
// numbers (zero, subnormals and non-finite values by the conversion).
__device__ __forceinline__ double f2d_exact(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xFFu;
    if (e == 0u || e == 0xFFu)
        return (double)f;
    return __longlong_as_double((long long)(((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                                            ((uint64_t)(b & 0x7FFFFFu) << 29)));
}

// x < 0 for the heights of this step (never -0: they start >= +0, and
// x - x and x + y round to +0) by the sign bit, on the integer pipe.
__device__ __forceinline__ bool dneg(double x) { return __double2hiint(x) < 0; }

// x >= y for non-negative binary64 values: their bit patterns order alike.
__device__ __forceinline__ bool dge_pos(double x, double y)
{
    return __double_as_longlong(x) >= __double_as_longlong(y);
}

__global__ void __launch_bounds__(kSedNT) sed_move_kernel(const InstDev *__restrict__ P, int32_t n_cells, int64_t n_slots,
                                                          int32_t nx, double dz, float dt32,
                                                          const double *__restrict__ zeta,
                                                          const int32_t *__restrict__ group,
                                                          const int32_t *__restrict__ id_of_slot,
                                                          uint32_t *__restrict__ key, uint32_t *__restrict__ val,
                                                          double *__restrict__ zeta_new, uint32_t *__restrict__ counts,
                                                          double *__restrict__ precip_part, int32_t cbase,
                                                          int32_t *__restrict__ emig)
{
    constexpr unsigned FULL = 0xFFFFFFFFu;
    __shared__ double s_pr[kSedNT / 32];
    const PairConsts C = pair_consts(P);
    const int lane = threadIdx.x & 31;
    const int64_t *__restrict__ gxi = P->xi;
    const double *__restrict__ gv = P->v;
    const int64_t stride = (int64_t)gridDim.x * kSedNT;
    double pr = 0.0;
    // warp-uniform trip count: every lane runs every round (shuffles, ballots)
    for (int64_t w0 = ((int64_t)blockIdx.x * kSedNT + (threadIdx.x & ~31)); w0 < n_slots; w0 += kSedU * stride) {
        int32_t id[kSedU], g[kSedU];
        int64_t x[kSedU];
        double vv[kSedU], zt[kSedU];
#pragma unroll
        for (int u = 0; u < kSedU; ++u) {
            const int64_t sl = w0 + u * stride + lane;
            const bool in = sl < n_slots;
            id[u] = in ? id_of_slot[sl] : -1;
            g[u] = in ? group[sl] : 0;
            x[u] = in ? gxi[sl] : 0;
            vv[u] = in ? gv[sl] : 1.0;
            zt[u] = in ? zeta[sl] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kSedU; ++u) {
            const int64_t sl = w0 + u * stride + lane;
            int32_t ng = -1; // -1: no SD in this slot
            if (id[u] >= 0) {
                double zn = 0.0;
                int32_t em = -1;
                ng = n_cells;
                if (g[u] < n_cells && x[u] > 0) {
                    bool in_range;
                    const float vf = d2f_rn(vv[u], in_range);
                    const double d = f2d_exact(__fmul_rn(vt32c(C, radius32(vf)), dt32));
                    double zz = __dsub_rn(zt[u], d);
                    // crossing k levels takes cell c to c - k nx; below the
                    // grid's level 0 exactly when cbase + c is negative
                    // (0 <= column < nx)
                    int32_t c = g[u];
                    while (dneg(zz)) { // at most as many levels as the SD falls through
                        c -= nx;
                        if (c + cbase < 0)
                            break;
                        zz = __dadd_rn(zz, dz);
                    }
                    if (c + cbase < 0) {
                        pr = __dadd_rn(pr, __dmul_rn(xi2d(x[u]), vv[u]));
                    } else {
                        if (dge_pos(zz, dz)) { // zeta + dz rounded up to dz: on the boundary, level above
                            c += nx;
                            zz = 0.0;
                        }
                        zn = zz;
                        if (c >= 0)
                            ng = c;
                        else // into another piece of the grid
                            em = c + cbase;
                    }
                }
                key[id[u]] = (uint32_t)ng;
                val[id[u]] = (uint32_t)sl;
                zeta_new[sl] = zn;
                emig[id[u]] = em;
            }
            const int32_t nxt = __shfl_down_sync(FULL, ng, 1);
            const bool end = lane == 31 || nxt != ng;
            const unsigned ends = __ballot_sync(FULL, end);
            if (end && ng >= 0) {
                const unsigned below = ends & ((1u << lane) - 1u);
                const int start = below ? 32 - __clz(below) : 0;
                atomicAdd(&counts[ng], (uint32_t)(lane - start + 1));
            }
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
        pr = __dadd_rn(pr, __shfl_down_sync(FULL, pr, d));
    if (lane == 0)
        s_pr[threadIdx.x >> 5] = pr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kSedNT / 32; ++w)
            t = __dadd_rn(t, s_pr[w]);
        precip_part[blockIdx.x] = t;
    }
}

// One block: ustart = exclusive scan of counts[0 .. n_groups) (total at
// ustart[n_groups]); poff the same with every count rounded up to even;
// *precip_total = sum of precip[0 .. n_parts) in a fixed order.  Both scans
// run at once on packed 64-bit sums (unpadded below, padded above: neither
// exceeds 2^31), 8 consecutive groups per thread, tiles of 8192 groups.
__global__ void __launch_bounds__(1024) sed_scan_kernel(const uint32_t *__restrict__ counts, int32_t n_groups,
                                                        int32_t *__restrict__ ustart, int32_t *__restrict__ poff,
                                                        const double *__restrict__ precip, int32_t n_parts,
                                                        double *__restrict__ precip_total)
{
    constexpr int E = 8, TILE = 1024 * E;
    __shared__ uint32_t s_c[TILE];
    __shared__ unsigned long long s_w[32];
    __shared__ double s_pr[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    unsigned long long carry = 0;
    for (int32_t g0 = 0; g0 < n_groups; g0 += TILE) {
        {
            uint32_t c[E]; // the tile's loads all in flight at once
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = t + e * 1024;
                c[e] = g0 + i < n_groups ? counts[g0 + i] : 0u;
            }
#pragma unroll
            for (int e = 0; e < E; ++e)
                s_c[t + e * 1024] = c[e];
        }
        __syncthreads();
        unsigned long long v[E], sum = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const uint32_t c = s_c[t * E + e];
            v[e] = (unsigned long long)c | ((unsigned long long)((c + 1u) & ~1u) << 32);
            sum += v[e];
        }
        unsigned long long x = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if (lane >= d)
                x += y;
        }
        if (lane == 31)
            s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = s_w[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, w, d);
                if (lane >= d)
                    w += y;
            }
            s_w[lane] = w; // inclusive totals of warps 0 .. lane
        }
        __syncthreads();
        // the two results through shared memory, so that the writes to
        // global memory are coalesced (consecutive threads, consecutive groups)
        const unsigned long long base0 = carry + (warp > 0 ? s_w[warp - 1] : 0ull) + x - sum;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            unsigned long long base = base0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                s_c[t * E + e] = (uint32_t)(half ? base >> 32 : base);
                base += v[e];
            }
            __syncthreads();
            int32_t *out = half ? poff : ustart;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int32_t g = g0 + t + e * 1024;
                if (g < n_groups)
                    out[g] = (int32_t)s_c[t + e * 1024];
            }
            __syncthreads();
        }
        carry += s_w[31];
    }
    if (t == 0) {
        ustart[n_groups] = (int32_t)(uint32_t)carry;
        poff[n_groups] = (int32_t)(uint32_t)(carry >> 32);
    }
    // the precipitated water: thread t sums parts t, t + 1024, ... in order,
    // then a fixed tree over the threads (the loads of four parts in flight
    // at once, the sums in the same order)
    double pr = 0.0;
    for (int i0 = t; i0 < n_parts; i0 += 4 * 1024) {
        double q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            q[u] = i0 + u * 1024 < n_parts ? precip[i0 + u * 1024] : 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + u * 1024 < n_parts)
                pr = __dadd_rn(pr, q[u]);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
        pr = __dadd_rn(pr, __shfl_down_sync(0xFFFFFFFFu, pr, d));
    if (lane == 0)
        s_pr[warp] = pr;
    __syncthreads();
    if (warp == 0) {
        pr = s_pr[lane];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1)
            pr = __dadd_rn(pr, __shfl_down_sync(0xFFFFFFFFu, pr, d));
        if (lane == 0)
            *precip_total = pr;
    }
}

// hist[d * n_tiles + tile] = keys of the tile whose digit (key >> shift) & 255 is d.
__global__ void __launch_bounds__(kRadixNT) radix_hist_kernel(const uint32_t *__restrict__ keys, int64_t n, int shift,
                                                              uint32_t *__restrict__ hist, int32_t n_tiles)
{
    __shared__ uint32_t h[kRadixBuckets];
    const int t = threadIdx.x;
    h[t] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    uint32_t k[kRadixRounds]; // every load of the thread in flight at once
#pragma unroll
    for (int r = 0; r < kRadixRounds; ++r) {
        const int64_t i = base + (int64_t)r * kRadixNT + t;
        k[r] = i < n ? keys[i] : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int r = 0; r < kRadixRounds; ++r)
        if (base + (int64_t)r * kRadixNT + t < n)
            atomicAdd(&h[(k[r] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(int64_t)t * n_tiles + blockIdx.x] = h[t];
}

// Block d: exclusive scan, in place, of the counts of digit d over the
// tiles (one contiguous row of hist), in chunks of 1024 with a running
// carry; total[d] = the row's sum.
__global__ void __launch_bounds__(1024) radix_row_scan_kernel(uint32_t *__restrict__ hist, int32_t n_tiles,
                                                              uint32_t *__restrict__ total)
{
    __shared__ uint32_t s[1024];
    __shared__ uint32_t s_warp[32];
    const int t = threadIdx.x;
    uint32_t *row = hist + (int64_t)blockIdx.x * n_tiles;
    uint32_t carry = 0;
    for (int32_t c0 = 0; c0 < n_tiles; c0 += 1024) {
        const int32_t i = c0 + t;
        s[t] = i < n_tiles ? row[i] : 0u;
        __syncthreads();
        const uint32_t sum = block_exclusive_scan<1024, 1024>(s, s_warp);
        if (i < n_tiles)
            row[i] = carry + s[t];
        carry += sum;
        __syncthreads();
    }
    if (t == 0)
        total[blockIdx.x] = carry;
}

// One block of 256: exclusive scan of the digit totals, in place.
__global__ void __launch_bounds__(kRadixBuckets) radix_digit_scan_kernel(uint32_t *__restrict__ total)
{
    __shared__ uint32_t s[kRadixBuckets];
    __shared__ uint32_t s_warp[32];
    s[threadIdx.x] = total[threadIdx.x];
    __syncthreads();
    block_exclusive_scan<kRadixBuckets, kRadixBuckets>(s, s_warp);
    total[threadIdx.x] = s[threadIdx.x];
}

// Stable scatter of one pass: tile keys in index order (round-major, thread
// minor); within a round, lanes of a warp with equal digits are ranked by
// __match_any_sync, warps by their per-digit counts in shared memory.
__global__ void __launch_bounds__(kRadixNT) radix_scatter_kernel(const uint32_t *__restrict__ keys_in,
                                                                 const uint32_t *__restrict__ vals_in, int64_t n,
                                                                 int shift, const uint32_t *__restrict__ offs,
                                                                 const uint32_t *__restrict__ digit_base,
                                                                 int32_t n_tiles, uint32_t *__restrict__ keys_out,
                                                                 uint32_t *__restrict__ vals_out)
{
    constexpr int NW = kRadixNT / 32;
    __shared__ uint32_t s_base[kRadixBuckets + 1];
    __shared__ uint32_t s_wcnt[NW][kRadixBuckets + 1];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    s_base[t] = digit_base[t] + offs[(int64_t)t * n_tiles + blockIdx.x];
    for (int i = t; i < NW * (kRadixBuckets + 1); i += kRadixNT)
        (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t kk[kRadixRounds], vv[kRadixRounds]; // every load of the thread in flight at once
#pragma unroll
    for (int r = 0; r < kRadixRounds; ++r) {
        const int64_t i = base + (int64_t)r * kRadixNT + t;
        kk[r] = i < n ? keys_in[i] : 0u;
        vv[r] = i < n ? vals_in[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kRadixRounds; ++r) {
        const int64_t i = base + (int64_t)r * kRadixNT + t;
        const bool valid = i < n;
        const uint32_t k = kk[r];
        const uint32_t v = vv[r];
        const uint32_t d = valid ? ((k >> shift) & 255u) : (uint32_t)kRadixBuckets;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t rank = (uint32_t)__popc(peers & lt);
        if (rank == 0)
            s_wcnt[warp][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t before = 0;
            for (int w = 0; w < warp; ++w)
                before += s_wcnt[w][d];
            const uint32_t pos = s_base[d] + before + rank;
            keys_out[pos] = k;
            vals_out[pos] = v;
        }
        __syncthreads();
        for (int dd = t; dd <= kRadixBuckets; dd += kRadixNT) {
            uint32_t sum = 0;
            for (int w = 0; w < NW; ++w) {
                sum += s_wcnt[w][dd];
                s_wcnt[w][dd] = 0;
            }
            if (dd < kRadixBuckets)
                s_base[dd] += sum;
        }
        __syncthreads();
    }
}

// The new layout: the j-th SD in (group, id) order goes to slot
// poff[g] + (j - ustart[g]).
__global__ void sed_gather_kernel(int64_t n_sd, const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                                  const int32_t *__restrict__ ustart, const int32_t *__restrict__ poff,
                                  const int64_t *__restrict__ xi, const double *__restrict__ v,
                                  const double *__restrict__ zeta_new, const int32_t *__restrict__ id_of_slot,
                                  int64_t *__restrict__ xi2, double *__restrict__ v2, double *__restrict__ zeta2,
                                  int32_t *__restrict__ id2, int32_t *__restrict__ group2)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_sd; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t g = keys[j], s = vals[j];
        const int64_t p = poff[g] + (j - ustart[g]);
        xi2[p] = xi[s];
        v2[p] = v[s];
        zeta2[p] = zeta_new[s];
        id2[p] = id_of_slot[s];
        group2[p] = (int32_t)g;
    }
}

// The padding slot after every odd group of the new layout.
__global__ void sed_pad_kernel(int32_t n_groups, const int32_t *__restrict__ ustart, const int32_t *__restrict__ poff,
                               int64_t *__restrict__ xi2, double *__restrict__ v2, double *__restrict__ zeta2,
                               int32_t *__restrict__ id2, int32_t *__restrict__ group2)
{
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n_groups; g += gridDim.x * blockDim.x) {
        for (int32_t p = poff[g] + (ustart[g + 1] - ustart[g]); p < poff[g + 1]; ++p) {
            xi2[p] = 0;
            v2[p] = 1.0;
            zeta2[p] = 0.0;
            id2[p] = -1;
            group2[p] = g;
        }
    }
}

// -------------------------------------------------------------------- host
// The second layout (swapped with the context's after every step, so both
// sets are freed through their current pointers) and the scratch.
struct SedBuffers {
    int64_t *xi2 = nullptr;
    double *v2 = nullptr;
    double *zeta2 = nullptr;
    int32_t *id2 = nullptr;
    int32_t *group = nullptr;     // group of every slot of the current layout
    int32_t *group2 = nullptr;
    int32_t *cell_off2 = nullptr; // n_cells + 2
    double *zeta_new = nullptr;   // per slot of the old layout
    uint32_t *keys[2] = {};
    uint32_t *vals[2] = {};
    uint32_t *counts = nullptr; // n_cells + 1
    int32_t *ustart = nullptr;  // n_cells + 2
    double *precip = nullptr;   // per-block parts of the move kernel, then the total
    uint32_t *hist = nullptr;   // 256 x tiles, then 256 digit totals
    uint32_t *flags = nullptr;  // flags, then the first bad id (8-byte aligned)
    int32_t *emig = nullptr;    // per SD id: its cell in another piece of the grid after the last step, or -1
    void *h_read = nullptr;     // pinned: the new offsets, the precipitated total and the plan's class counts
    cudaStream_t side = nullptr; // the offset scan (and the plan's refresh) beside the radix sort
    cudaEvent_t fork = nullptr, join = nullptr;
};

// Bytes of the pinned read-back buffer for n_cells cells: n_cells + 2
// offsets, the precipitated total (8-byte aligned) and 8 class-count words.
size_t sed_read_bytes(int32_t n_cells) { return (((size_t)n_cells + 2) * 4 + 7) / 8 * 8 + 8 + 32; }

void sed_release(sdm_ctx *ctx)
{
    if (ctx->sed) {
        SedBuffers &b = *ctx->sed;
        void *bufs[] = {b.xi2,      b.v2,       b.zeta2,    b.id2,    b.group,  b.group2,
                        b.cell_off2, b.zeta_new, b.keys[0], b.keys[1], b.vals[0], b.vals[1],
                        b.counts,   b.ustart,   b.precip,   b.hist,   b.flags,  b.emig};
        for (void *p : bufs)
            ctx->mem.put(p, 0);
        if (b.h_read || b.side) {
            cudaStreamSynchronize(ctx->stream); // no read-back in flight, the side stream joined
            if (b.side)
                cudaStreamSynchronize(b.side);
        }
        if (b.h_read)
            cudaFreeHost(b.h_read);
        if (b.side)
            cudaStreamDestroy(b.side);
        if (b.fork)
            cudaEventDestroy(b.fork);
        if (b.join)
            cudaEventDestroy(b.join);
        delete ctx->sed;
        ctx->sed = nullptr;
    }
    ctx->mem.put(ctx->d_zeta, 0);
    ctx->d_zeta = nullptr;
}

template <typename T>
T *sed_get(sdm_ctx *ctx, size_t count)
{
    return static_cast<T *>(ctx->mem.get(sizeof(T) * (count > 0 ? count : 1)));
}

sdm_status sed_alloc(sdm_ctx *ctx)
{
    if (ctx->sed)
        return SDM_OK;
    ctx->sed = new (std::nothrow) SedBuffers();
    if (!ctx->sed)
        return fail(&ctx->error, SDM_ENOMEM, "host allocation failed");
    SedBuffers &b = *ctx->sed;
    const int64_t slots = ctx->n_slots_cap, cap = ctx->capacity_sd;
    const int32_t nc = ctx->cfg.n_cells;
    const int64_t tiles = (cap + kRadixTile - 1) / kRadixTile;
    ctx->d_zeta = (double *)ctx->mem.get(sizeof(double) * slots);
    b.xi2 = sed_get<int64_t>(ctx, slots);
    b.v2 = sed_get<double>(ctx, slots);
    b.zeta2 = sed_get<double>(ctx, slots);
    b.id2 = sed_get<int32_t>(ctx, slots);
    b.group = sed_get<int32_t>(ctx, slots);
    b.group2 = sed_get<int32_t>(ctx, slots);
    b.cell_off2 = sed_get<int32_t>(ctx, (size_t)nc + 2);
    b.zeta_new = sed_get<double>(ctx, slots);
    for (int i = 0; i < 2; ++i) {
        b.keys[i] = sed_get<uint32_t>(ctx, cap);
        b.vals[i] = sed_get<uint32_t>(ctx, cap);
    }
    b.counts = sed_get<uint32_t>(ctx, (size_t)nc + 1);
    b.ustart = sed_get<int32_t>(ctx, (size_t)nc + 2);
    b.precip = sed_get<double>(ctx, (size_t)kSedMaxBlocks + 1);
    b.hist = sed_get<uint32_t>(ctx, (size_t)kRadixBuckets * tiles + kRadixBuckets);
    b.flags = sed_get<uint32_t>(ctx, 4);
    b.emig = sed_get<int32_t>(ctx, cap);
    if (cudaMallocHost(&b.h_read, sed_read_bytes(nc)) != cudaSuccess) {
        cudaGetLastError();
        b.h_read = nullptr;
    }
    if (cudaStreamCreateWithFlags(&b.side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        sed_release(ctx);
        return fail(&ctx->error, SDM_ENOMEM, "sedimentation stream and events: creation failed");
    }
    const bool ok = ctx->d_zeta && b.xi2 && b.v2 && b.zeta2 && b.id2 && b.group && b.group2 && b.cell_off2 &&
                    b.zeta_new && b.keys[0] && b.keys[1] && b.vals[0] && b.vals[1] && b.counts && b.ustart &&
                    b.precip && b.hist && b.flags && b.emig && b.h_read;
    if (!ok) {
        sed_release(ctx);
        return fail(&ctx->error, SDM_ENOMEM, "sedimentation buffers: device allocation failed");
    }
    ctx->device_bytes += slots * (8 + 8 + 8 + 8 + 4 + 4 + 4 + 8) + cap * 20 + ((int64_t)nc + 2) * 16 +
                         (int64_t)kRadixBuckets * (tiles + 1) * 4;
    return SDM_OK;
}

int sed_grid(int32_t n_groups)
{
    return std::max(1, std::min((n_groups + kSedNT / 32 - 1) / (kSedNT / 32), 152 * 16));
}

} // namespace

namespace {

// sdm_set_positions (zeta_in = 0: z above the grid's bottom) and
// sdm_set_heights (zeta_in = 1: z holds the heights above the cells' bottoms)
sdm_status set_positions_impl(sdm_ctx *ctx, const double *z, int32_t nx, double dz, int on_device, int zeta_in)
{
    sdm_status st = ctx_usable(ctx);
    if (st != SDM_OK)
        return st;
    if (!ctx->has_attributes)
        return fail(&ctx->error, SDM_ESTATE, "sdm_set_attributes has not been called");
    const int32_t nc = ctx->cfg.n_cells;
    if (!z || nx < 1 || nc % nx != 0 || !(std::isfinite(dz) && dz > 0.0))
        return fail(&ctx->error, SDM_EINVAL, "need z, nx >= 1 dividing n_cells = %d, and a finite dz > 0", nc);
    if (ctx->cfg.cell_base % nx != 0)
        return fail(&ctx->error, SDM_EINVAL, "nx = %d must divide cell_base = %d (pieces of a grid are whole levels)",
                    nx, ctx->cfg.cell_base);
    st = sed_alloc(ctx);
    if (st != SDM_OK)
        return st;
    cudaStream_t s = ctx->stream;
    const double *dz_arr = z;
    void *stage = nullptr;
    const size_t bz = sizeof(double) * ctx->n_sd;
    if (!on_device) {
        stage = ctx->mem.get(bz);
        if (!stage)
            return fail(&ctx->error, SDM_ENOMEM, "staging allocation failed");
        CTX_CUDA(ctx, cudaMemcpyAsync(stage, z, bz, cudaMemcpyHostToDevice, s));
        dz_arr = (const double *)stage;
    }
    uint32_t *d_flags = ctx->sed->flags;
    unsigned long long *d_bad = (unsigned long long *)(d_flags + 2);
    CTX_CUDA(ctx, cudaMemsetAsync(d_flags, 0, sizeof(uint32_t), s));
    CTX_CUDA(ctx, cudaMemsetAsync(d_bad, 0xFF, sizeof(unsigned long long), s));
    sed_set_kernel<<<sed_grid(nc + 1), kSedNT, 0, s>>>(ctx->d_cell_off, nc, ctx->n_slots, ctx->d_id_of_slot, dz_arr,
                                                        nx, dz, ctx->cfg.cell_base, zeta_in, ctx->d_zeta,
                                                        ctx->sed->group, d_flags, d_bad);
    CTX_CUDA(ctx, cudaMemsetAsync(ctx->sed->emig, 0xFF, sizeof(int32_t) * ctx->n_sd, s));
    uint32_t flags = 0;
    unsigned long long bad = 0;
    CTX_CUDA(ctx, cudaGetLastError());
    CTX_CUDA(ctx, cudaMemcpyAsync(&flags, d_flags, sizeof flags, cudaMemcpyDeviceToHost, s));
    CTX_CUDA(ctx, cudaMemcpyAsync(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost, s));
    CTX_CUDA(ctx, cudaStreamSynchronize(s));
    ctx->mem.put(stage, bz);
    if (flags & 1u) {
        ctx->has_positions = false;
        return fail(&ctx->error, SDM_EINVAL,
                    zeta_in ? "SD %llu: zeta must lie in [0, dz)" : "SD %llu: z must lie in its cell's level [iz dz, (iz + 1) dz)",
                    bad);
    }
    ctx->nx = nx;
    ctx->dz = dz;
    ctx->has_positions = true;
    return SDM_OK;
}

} // namespace

extern "C" sdm_status sdm_set_positions(sdm_ctx *ctx, const double *z, int32_t nx, double dz, int on_device)
{
    NvtxRange nvtx_range("sdm_set_positions");
    return set_positions_impl(ctx, z, nx, dz, on_device, 0);
}

extern "C" sdm_status sdm_set_heights(sdm_ctx *ctx, const double *zeta, int32_t nx, double dz, int on_device)
{
    NvtxRange nvtx_range("sdm_set_heights");
    return set_positions_impl(ctx, zeta, nx, dz, on_device, 1);
}

extern "C" sdm_status sdm_sedimentation_step(sdm_ctx *ctx, double *precipitated)
{
    NvtxRange nvtx_range("sdm_sedimentation_step");
    sdm_status st = ctx_usable(ctx);
    if (st != SDM_OK)
        return st;
    if (!ctx->has_attributes || !ctx->has_positions)
        return fail(&ctx->error, SDM_ESTATE, "sdm_set_positions has not been called for the current attributes");
    SedBuffers &b = *ctx->sed;
    cudaStream_t s = ctx->stream;
    const int32_t nc = ctx->cfg.n_cells, n_groups = nc + 1;
    const int64_t n = ctx->n_sd;
    CTX_CUDA(ctx, cudaMemsetAsync(b.counts, 0, sizeof(uint32_t) * n_groups, s));
    const int move_blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>(kSedMaxBlocks, (ctx->n_slots + (int64_t)kSedNT * kSedU - 1) / ((int64_t)kSedNT * kSedU)));
    sed_move_kernel<<<move_blocks, kSedNT, 0, s>>>(ctx->d_inst, nc, ctx->n_slots, ctx->nx, ctx->dz, (float)ctx->cfg.dt,
                                                   ctx->d_zeta, b.group, ctx->d_id_of_slot, b.keys[0], b.vals[0],
                                                   b.zeta_new, b.counts, b.precip, ctx->cfg.cell_base, b.emig);
    // the offset scan, the refresh of the context's own launch plan (when
    // refreshable: rebuilt on the device for the new layout) and the read-back
    // into the pinned buffer (offsets, precipitated total, class counts) on
    // the side stream, beside the radix sort, which needs none of them
    sdm_batch *sb = ctx->self_batch;
    const bool refresh = sb && sb->plan.refreshable && same_tuning(sb->plan.tuning, current_tuning());
    unsigned char *hr = static_cast<unsigned char *>(b.h_read);
    const int32_t *off = reinterpret_cast<const int32_t *>(hr);
    const size_t at_pr = (((size_t)nc + 2) * 4 + 7) / 8 * 8;
    const uint32_t *rc = reinterpret_cast<const uint32_t *>(hr + at_pr + 8);
    CTX_CUDA(ctx, cudaEventRecord(b.fork, s));
    CTX_CUDA(ctx, cudaStreamWaitEvent(b.side, b.fork, 0));
    sed_scan_kernel<<<1, 1024, 0, b.side>>>(b.counts, n_groups, b.ustart, b.cell_off2, b.precip, move_blocks,
                                            b.precip + kSedMaxBlocks);
    // the new layout's padding slots (the gather writes only the others)
    sed_pad_kernel<<<(n_groups + 255) / 256, 256, 0, b.side>>>(n_groups, b.ustart, b.cell_off2, b.xi2, b.v2, b.zeta2,
                                                                b.id2, b.group2);
    if (refresh) {
        CTX_CUDA(ctx, plan_refresh(sb->plan, b.cell_off2, nc, ctx->cfg.cell_base, b.side));
        CTX_CUDA(ctx, cudaMemcpyAsync(hr + at_pr + 8, sb->plan.d_refresh, sizeof(uint32_t) * (kNumClass + 1),
                                      cudaMemcpyDeviceToHost, b.side));
    }
    CTX_CUDA(ctx, cudaMemcpyAsync(hr, b.cell_off2, sizeof(int32_t) * (n_groups + 1), cudaMemcpyDeviceToHost, b.side));
    CTX_CUDA(ctx, cudaMemcpyAsync(hr + at_pr, b.precip + kSedMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, b.side));
    CTX_CUDA(ctx, cudaEventRecord(b.join, b.side));
    // stable sort of the new groups, SD-id order in
    const int bits = 32 - __builtin_clz((unsigned)nc | 1u);
    const int passes = (bits + 7) / 8;
    const int32_t tiles = (int32_t)((n + kRadixTile - 1) / kRadixTile);
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        uint32_t *digit_total = b.hist + (size_t)kRadixBuckets * tiles;
        radix_hist_kernel<<<tiles, kRadixNT, 0, s>>>(b.keys[cur], n, 8 * p, b.hist, tiles);
        radix_row_scan_kernel<<<kRadixBuckets, 1024, 0, s>>>(b.hist, tiles, digit_total);
        radix_digit_scan_kernel<<<1, kRadixBuckets, 0, s>>>(digit_total);
        radix_scatter_kernel<<<tiles, kRadixNT, 0, s>>>(b.keys[cur], b.vals[cur], n, 8 * p, b.hist, digit_total,
                                                         tiles, b.keys[cur ^ 1], b.vals[cur ^ 1]);
        cur ^= 1;
    }
    CTX_CUDA(ctx, cudaStreamWaitEvent(s, b.join, 0));
    sed_gather_kernel<<<1216, 256, 0, s>>>(n, b.keys[cur], b.vals[cur], b.ustart, b.cell_off2, ctx->d_xi, ctx->d_v,
                                           b.zeta_new, ctx->d_id_of_slot, b.xi2, b.v2, b.zeta2, b.id2, b.group2);
    CTX_CUDA(ctx, cudaGetLastError());
    CTX_CUDA(ctx, cudaStreamSynchronize(s));
    double precip = 0.0;
    std::memcpy(&precip, hr + at_pr, sizeof precip);
    // the new layout becomes the state; the old one the next scratch
    std::swap(ctx->d_xi, b.xi2);
    std::swap(ctx->d_v, b.v2);
    std::swap(ctx->d_zeta, b.zeta2);
    std::swap(ctx->d_id_of_slot, b.id2);
    std::swap(ctx->d_cell_off, b.cell_off2);
    std::swap(b.group, b.group2);
    int32_t largest = 0;
    for (int32_t c = 0; c < nc; ++c)
        largest = std::max(largest, off[c + 1] - off[c]);
    const bool keep_plan = ctx->self_batch && ctx->h_cell_off.size() == (size_t)nc + 1 &&
                           std::equal(ctx->h_cell_off.begin(), ctx->h_cell_off.end(), off) &&
                           same_tuning(ctx->self_batch->plan.tuning, current_tuning());
    ctx->h_cell_off.assign(off, off + nc + 1);
    ctx->n_slots = off[n_groups];
    ctx->largest_cell = largest;
    ctx->layout_version += 1;
    ctx->dev_base = ctx->step;
    InstDev inst = make_inst(ctx);
    CTX_CUDA(ctx, cudaMemcpyAsync(ctx->d_inst, &inst, sizeof inst, cudaMemcpyHostToDevice, s));
    const bool refreshed = refresh && !keep_plan && rc[kNumClass] == 0;
    if (refreshed)
        for (int k = 0; k < kNumClass; ++k)
            ctx->self_batch->plan.n_items[k] = (int)rc[k];
    if (ctx->self_batch && (keep_plan || refreshed))
        ctx->self_batch->versions[0] = ctx->layout_version;
    if (ctx->self_batch && !keep_plan && !refreshed) {
        batch_release(ctx->self_batch);
        delete ctx->self_batch;
        ctx->self_batch = nullptr;
    }
    if (precipitated)
        *precipitated = precip;
    return SDM_OK;
}

extern "C" sdm_status sdm_get_positions(sdm_ctx *ctx, double *z, int32_t *cell, int on_device)
{
    NvtxRange nvtx_range("sdm_get_positions");
    sdm_status st = ctx_usable(ctx);
    if (st != SDM_OK)
        return st;
    if (!ctx->has_attributes)
        return fail(&ctx->error, SDM_ESTATE, "sdm_set_attributes has not been called");
    if (z && !ctx->has_positions)
        return fail(&ctx->error, SDM_ESTATE, "no positions: sdm_set_positions has not been called");
    if (!z && !cell)
        return SDM_OK;
    cudaStream_t s = ctx->stream;
    const int32_t nc = ctx->cfg.n_cells;
    const int32_t nx = ctx->has_positions ? ctx->nx : 1;
    const int64_t n = ctx->n_sd;
    if (on_device) {
        sed_get_kernel<<<sed_grid(nc + 1), kSedNT, 0, s>>>(ctx->d_cell_off, nc, ctx->n_slots, ctx->d_id_of_slot,
                                                            ctx->d_zeta, nx, ctx->dz, ctx->cfg.cell_base, nullptr, z,
                                                            cell, nullptr, nullptr);
        CTX_CUDA(ctx, cudaGetLastError());
        return SDM_OK;
    }
    const size_t bz = sizeof(double) * n, bc = sizeof(int32_t) * n;
    char *tmp = (char *)ctx->mem.get(bz + bc);
    if (!tmp)
        return fail(&ctx->error, SDM_ENOMEM, "allocation failed");
    sed_get_kernel<<<sed_grid(nc + 1), kSedNT, 0, s>>>(ctx->d_cell_off, nc, ctx->n_slots, ctx->d_id_of_slot,
                                                        ctx->d_zeta, nx, ctx->dz, ctx->cfg.cell_base, nullptr,
                                                        z ? (double *)tmp : nullptr,
                                                        cell ? (int32_t *)(tmp + bz) : nullptr, nullptr, nullptr);
    CTX_CUDA(ctx, cudaGetLastError());
    if (z)
        CTX_CUDA(ctx, cudaMemcpyAsync(z, tmp, bz, cudaMemcpyDeviceToHost, s));
    if (cell)
        CTX_CUDA(ctx, cudaMemcpyAsync(cell, tmp + bz, bc, cudaMemcpyDeviceToHost, s));
    CTX_CUDA(ctx, cudaStreamSynchronize(s));
    ctx->mem.put(tmp, bz + bc);
    return check_device_status(ctx);
}

extern "C" sdm_status sdm_get_heights(sdm_ctx *ctx, double *zeta, int32_t *cell, int on_device)
{
    NvtxRange nvtx_range("sdm_get_heights");
    sdm_status st = ctx_usable(ctx);
    if (st != SDM_OK)
        return st;
    if (!ctx->has_attributes || !ctx->has_positions)
        return fail(&ctx->error, SDM_ESTATE, "no positions: sdm_set_positions has not been called");
    if (!zeta && !cell)
        return SDM_OK;
    cudaStream_t s = ctx->stream;
    const int32_t nc = ctx->cfg.n_cells;
    const int64_t n = ctx->n_sd;
    const int32_t *emig = ctx->sed->emig;
    if (on_device) {
        sed_get_kernel<<<sed_grid(nc + 1), kSedNT, 0, s>>>(ctx->d_cell_off, nc, ctx->n_slots, ctx->d_id_of_slot,
                                                            ctx->d_zeta, ctx->nx, ctx->dz, ctx->cfg.cell_base, emig,
                                                            nullptr, nullptr, zeta, cell);
        CTX_CUDA(ctx, cudaGetLastError());
        return SDM_OK;
    }
    const size_t bz = sizeof(double) * n, bc = sizeof(int32_t) * n;
    char *tmp = (char *)ctx->mem.get(bz + bc);
    if (!tmp)
        return fail(&ctx->error, SDM_ENOMEM, "allocation failed");
    sed_get_kernel<<<sed_grid(nc + 1), kSedNT, 0, s>>>(ctx->d_cell_off, nc, ctx->n_slots, ctx->d_id_of_slot,
                                                        ctx->d_zeta, ctx->nx, ctx->dz, ctx->cfg.cell_base, emig, nullptr,
                                                        nullptr, zeta ? (double *)tmp : nullptr,
                                                        cell ? (int32_t *)(tmp + bz) : nullptr);
    CTX_CUDA(ctx, cudaGetLastError());
    if (zeta)
        CTX_CUDA(ctx, cudaMemcpyAsync(zeta, tmp, bz, cudaMemcpyDeviceToHost, s));
    if (cell)
        CTX_CUDA(ctx, cudaMemcpyAsync(cell, tmp + bz, bc, cudaMemcpyDeviceToHost, s));
    CTX_CUDA(ctx, cudaStreamSynchronize(s));
    ctx->mem.put(tmp, bz + bc);
    return check_device_status(ctx);
}
