// Kernels of the SDM coalescence step on sm_103a.
//
//  cell_step_kernel<CAP, NT>   one CTA per cell of at most CAP stored SDs:
//      16-byte vector loads of xi and v into shared memory, in-kernel Philox
//      sort keys, a one-pass shared-memory bucket sort (keys are uniform, so
//      bucketing on the top log2(CAP) bits leaves ~1 key per bucket and a
//      short comparison fix-up finishes the order), pairing, the filtered
//      collision count, and stores of changed SDs only.
//  big_*_kernel                cells above the shared-memory capacity: a
//      histogram pass over chunks, a per-cell scan, a scatter of (key, rank)
//      into bucket order in global scratch, a per-bucket shared-memory sort
//      on the next key bits, and a pair pass gathering from the state.
//  spectrum kernels            dv/dlnr accumulation per cell, or in total
//                              without atomics (fixed summation order).
//  layout / gather kernels     set_attributes and get_attributes.
#pragma once

#include "sdm_device.cuh"

namespace sdm {

constexpr int ilog2_c(int x) { return x <= 1 ? 0 : 1 + ilog2_c(x / 2); }

// Exclusive scan, in place, of s[0 .. NITEMS) by NT threads; returns the
// total to every thread.  Ends with the block synchronised.
template <int NT, int NITEMS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t *s, uint32_t *s_warp)
{
    constexpr int E = (NITEMS + NT - 1) / NT;
    constexpr int NW = NT / 32;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t loc[E];
    uint32_t sum = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int idx = t * E + e;
        loc[e] = idx < NITEMS ? s[idx] : 0u;
        sum += loc[e];
    }
    uint32_t x = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= d)
            x += y;
    }
    if (lane == 31)
        s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? s_warp[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, d);
            if (lane >= d)
                w += y;
        }
        if (lane < NW)
            s_warp[lane] = w;
    }
    __syncthreads();
    uint32_t base = (warp > 0 ? s_warp[warp - 1] : 0u) + x - sum;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int idx = t * E + e;
        if (idx < NITEMS)
            s[idx] = base;
        base += loc[e];
    }
    const uint32_t total = s_warp[NW - 1];
    __syncthreads();
    return total;
}

__device__ __forceinline__ bool key_less(uint64_t ka, uint32_t ra, uint64_t kb, uint32_t rb)
{
    return (ka < kb) | ((ka == kb) & (ra < rb));
}

// ------------------------------------------------- bulk copies, mbarriers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Global -> shared bulk copy through the TMA engine, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Bounded wait on an mbarrier phase: ~2^22 polls (each poll may suspend the
// thread for a hardware-defined interval), then give up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t max_polls = 1u << 22)
{
    for (uint32_t it = 0; it < max_polls; ++it)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

// The bounded-wait path on its own: a barrier that expects two arrivals gets
// one, so its phase never completes; lane 0 waits at most max_polls polls
// and records whether it gave up (1) or saw the phase complete (0).
__global__ void selftest_wait_kernel(uint32_t max_polls, uint32_t *out)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
        out[0] = mbar_wait_bounded(&bar, 0u, max_polls) ? 0u : 1u;
    }
}

// -------------------------------------------------------------- cell step
// A pair the filter could not decide, waiting for the exact evaluation.
struct QEntry {
    int64_t xj, xk;
    double vj, vk;
    uint32_t slot_j, slot_k; // storage slots in the run's arrays
    uint32_t wa, wb;         // the pair's uniform words
    uint32_t n_c;            // live SDs of its cell
    int32_t inst;            // its run
    int32_t gamma;           // certain collision count (>= 1), or -1: evaluate exactly
    int32_t pad_;
};

constexpr int kQueueFlush = 64; // flush once this many pairs wait

template <int CAP>
struct QueueCap {
    static constexpr int value = (kQueueFlush + CAP / 2) < 512 ? (kQueueFlush + CAP / 2) : 512;
};

template <int CAP, int STAGES>
struct CellSmem {
    // STAGES x (xi, v) staging + key, bucket, rank, perm work arrays + queue
    static constexpr size_t bytes =
        (size_t)CAP * (16 * STAGES + 8 + 4 + 2 + 2) + sizeof(QEntry) * (size_t)QueueCap<CAP>::value;
};

// Persistent: CTA b handles work items b, b + gridDim.x, ...  Thread 0
// streams the next STAGES - 1 cells into shared memory with bulk copies
// while the CTA works on the current one.  Pairs the binary32 filter cannot
// decide wait in a shared-memory queue (across cells) and are evaluated
// exactly, one per lane, when kQueueFlush of them have gathered and at the
// end: every SD belongs to one pair per step and nothing reads it again in
// this launch, so deferring its update is safe.
template <int CAP, int NT, int STAGES>
__global__ void __launch_bounds__(NT, (1024 / NT > 0 ? 1024 / NT : 1)) cell_step_kernel(const WorkItem *__restrict__ items, int32_t n_items,
                                                       InstDev *const *__restrict__ insts, int64_t step_offset)
{
    constexpr int NB = CAP;
    constexpr int LB = ilog2_c(CAP);
    constexpr int RP = (CAP / 2 + NT - 1) / NT; // rank pairs per thread
    static_assert((1 << LB) == CAP, "CAP must be a power of two");
    static_assert(CAP <= 65536, "ranks are stored in 16 bits");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    int64_t *st_xi = reinterpret_cast<int64_t *>(smem_raw);          // [STAGES][CAP]
    double *st_v = reinterpret_cast<double *>(st_xi + STAGES * CAP); // [STAGES][CAP]
    uint64_t *s_key = reinterpret_cast<uint64_t *>(st_v + STAGES * CAP);
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(s_key + CAP);
    uint16_t *s_rank = reinterpret_cast<uint16_t *>(s_hist + NB);
    uint16_t *s_perm = s_rank + CAP;
    QEntry *s_q = reinterpret_cast<QEntry *>(s_perm + CAP);
    constexpr uint32_t QCAP = QueueCap<CAP>::value;
    __shared__ uint32_t s_qn;
    __shared__ uint64_t s_bar[STAGES];
    __shared__ int4 s_meta[STAGES]; // off, n, cell, inst
    __shared__ uint32_t s_warp[32];

    const int t = threadIdx.x;
    if (t == 0) {
        for (int i = 0; i < STAGES; ++i)
            mbar_init(&s_bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_qn = 0;
    }
    __syncthreads();

    auto flush = [&]() { // all threads; the queue's contents are visible to all
        const uint32_t nq = s_qn < QCAP ? s_qn : QCAP;
        for (uint32_t e = t; e < nq; e += NT) {
            QEntry E = s_q[e];
            InstDev *Pq = insts[E.inst];
            const int64_t g = E.gamma > 0 ? cap_gamma(E.gamma, E.xj, E.xk)
                                          : pair_gamma_exact(Pq, E.n_c, E.xj, E.xk, E.vj, E.vk, E.wa, E.wb);
            if (g > 0) {
                const bool split = shima_update(g, E.xj, E.xk, E.vj, E.vk);
                Pq->xi[E.slot_j] = E.xj;
                Pq->xi[E.slot_k] = E.xk;
                Pq->v[E.slot_k] = E.vk;
                if (split)
                    Pq->v[E.slot_j] = E.vj;
            }
        }
        __syncthreads();
        if (t == 0)
            s_qn = 0;
        __syncthreads();
    };

    auto issue = [&](int k) { // thread 0: start loading the k-th cell of this CTA
        const int i = blockIdx.x + k * gridDim.x;
        if (i >= n_items)
            return;
        const int sg = k % STAGES;
        const WorkItem it = items[i];
        const InstDev *P = insts[it.inst];
        s_meta[sg] = make_int4(it.off, it.n, it.cell, it.inst);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&s_bar[sg], (uint32_t)it.n * 16u);
        bulk_g2s(st_xi + sg * CAP, P->xi + it.off, (uint32_t)it.n * 8u, &s_bar[sg]);
        bulk_g2s(st_v + sg * CAP, P->v + it.off, (uint32_t)it.n * 8u, &s_bar[sg]);
    };
    if (t == 0)
        for (int k = 0; k < STAGES - 1; ++k)
            issue(k);

    for (int k = 0; blockIdx.x + k * gridDim.x < n_items; ++k) {
        if (t == 0)
            issue(k + STAGES - 1);
        const int sg = k % STAGES;
        const bool arrived = mbar_wait_bounded(&s_bar[sg], (uint32_t)(k / STAGES) & 1u);
        if (!__syncthreads_and(arrived)) {
            // a copy never completed: report, wait (bounded) for the copies
            // still in flight, leave
            if (t == 0) {
                atomicOr(&insts[s_meta[sg].w]->status, 1u);
                for (int kk = k; kk < k + STAGES; ++kk) // copies issued and not consumed
                    if (blockIdx.x + kk * gridDim.x < n_items)
                        mbar_wait_bounded(&s_bar[kk % STAGES], (uint32_t)(kk / STAGES) & 1u);
            }
            return;
        }
        const int4 meta = s_meta[sg];
        const int n = meta.y;
        const uint32_t cell = (uint32_t)meta.z;
        InstDev *__restrict__ P = insts[meta.w];
        const int64_t s = P->step + step_offset;
        const uint64_t seed = P->seed;
        const int64_t *xs = st_xi + sg * CAP;
        const double *vs = st_v + sg * CAP;
        int64_t *__restrict__ gxi = P->xi + meta.x;
        double *__restrict__ gv = P->v + meta.x;

        for (int i = t; i < NB; i += NT)
            s_hist[i] = 0u;
        __syncthreads();

        // sort keys of live SDs and their bucket slots
        uint64_t key[2 * RP];
        uint32_t slot[2 * RP];
#pragma unroll
        for (int r = 0; r < RP; ++r) {
            const int q = t + r * NT;
            slot[2 * r] = 0xFFFFFFFFu;
            slot[2 * r + 1] = 0xFFFFFFFFu;
            key[2 * r] = 0;
            key[2 * r + 1] = 0;
            if (2 * q < n) {
                const bool la = xs[2 * q] > 0, lb = xs[2 * q + 1] > 0;
                if (la | lb) {
                    const uint4 w = draw4(seed, (uint32_t)q, cell, s, 0u);
                    if (la) {
                        key[2 * r] = ((uint64_t)w.x << 32) | w.y;
                        slot[2 * r] = atomicAdd(&s_hist[key[2 * r] >> (64 - LB)], 1u);
                    }
                    if (lb) {
                        key[2 * r + 1] = ((uint64_t)w.z << 32) | w.w;
                        slot[2 * r + 1] = atomicAdd(&s_hist[key[2 * r + 1] >> (64 - LB)], 1u);
                    }
                }
            }
        }
        __syncthreads();

        // bucket starts; the total is the live count n_c
        const uint32_t n_c = block_exclusive_scan<NT, NB>(s_hist, s_warp);
        if (n_c >= 2) {
            // scatter into bucket order
#pragma unroll
            for (int r = 0; r < RP; ++r) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (slot[2 * r + h] != 0xFFFFFFFFu) {
                        const uint32_t pos = s_hist[key[2 * r + h] >> (64 - LB)] + slot[2 * r + h];
                        s_key[pos] = key[2 * r + h];
                        s_rank[pos] = (uint16_t)(2 * (t + r * NT) + h);
                    }
                }
            }
            __syncthreads();

            // order within each bucket by (key, rank)
            for (uint32_t pos = t; pos < n_c; pos += NT) {
                const uint64_t kk = s_key[pos];
                const uint32_t rk = s_rank[pos];
                const uint32_t b = (uint32_t)(kk >> (64 - LB));
                const uint32_t lo = s_hist[b];
                const uint32_t hi = (b + 1 < (uint32_t)NB) ? s_hist[b + 1] : n_c;
                uint32_t cnt = 0;
                for (uint32_t m = lo; m < hi; ++m)
                    cnt += key_less(s_key[m], s_rank[m], kk, rk) ? 1u : 0u;
                s_perm[lo + cnt] = (uint16_t)rk;
            }
            __syncthreads();

            // pairs (l = 2q, 2q + 1 share one Philox block): the filter
            // settles almost all; the rest join the queue
            const uint32_t n_pairs = n_c / 2;
            const float ratio_f = u32_to_f32_rn((n_c & 1u) ? n_c : n_c - 1u);
            const PairConsts C = pair_consts(P);
            for (uint32_t q = t; 2 * q < n_pairs; q += NT) {
                const uint4 w = draw4(seed, q, cell, s, 1u);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t l = 2 * q + h;
                    if (l >= n_pairs)
                        break;
                    int a = s_perm[2 * l], b = s_perm[2 * l + 1];
                    int64_t xa = xs[a], xb = xs[b];
                    if (xa < xb) { // j holds the larger multiplicity; ties keep the earlier
                        const int tmp = a;
                        a = b;
                        b = tmp;
                        const int64_t tx = xa;
                        xa = xb;
                        xb = tx;
                    }
                    double va = vs[a], vb = vs[b];
                    const uint32_t wa = h ? w.z : w.x, wb = h ? w.w : w.y;
                    const int32_t gf = pair_gamma_filter(C, ratio_f, xa, va, vb, wa);
                    if (gf == 0)
                        continue;
                    const uint32_t qi = atomicAdd(&s_qn, 1u);
                    if (qi < QCAP) {
                        QEntry E;
                        E.xj = xa;
                        E.xk = xb;
                        E.vj = va;
                        E.vk = vb;
                        E.slot_j = (uint32_t)(meta.x + a);
                        E.slot_k = (uint32_t)(meta.x + b);
                        E.wa = wa;
                        E.wb = wb;
                        E.n_c = n_c;
                        E.inst = meta.w;
                        E.gamma = gf;
                        s_q[qi] = E;
                    } else { // queue full: update here
                        const int64_t g = gf > 0 ? cap_gamma(gf, xa, xb)
                                                 : pair_gamma_exact(P, n_c, xa, xb, va, vb, wa, wb);
                        if (g > 0) {
                            const bool split = shima_update(g, xa, xb, va, vb);
                            gxi[a] = xa;
                            gxi[b] = xb;
                            gv[b] = vb;
                            if (split)
                                gv[a] = va;
                        }
                    }
                }
            }
        }
        __syncthreads(); // stage sg and the work arrays are free again
        if (s_qn >= (uint32_t)kQueueFlush)
            flush();
    }
    if (s_qn > 0)
        flush();
}

// ------------------------------------------------------ warp-per-cell step
// Cells of at most 512 stored SDs: one warp per cell, no block barriers.
// Each warp runs its own bulk-copy pipeline (STAGES deep, one mbarrier per
// stage) and sorts its cell with a one-pass bucket sort (a warp scan of the
// bucket counts) and a register sort.  A pair the binary32 filter cannot
// decide is evaluated exactly at once, from the staged copy of its cell
// (every SD is in one pair per step, so nothing else in the launch reads or
// writes it).  No queue of such pairs is kept: that leaves 10.5 KB of shared
// memory per warp at 256 SDs, and 10 blocks of 2 warps per SM.
template <int CAP, int STAGES>
struct WarpSmem {
    // per warp: STAGES x (xi, v), sort word, bucket, perm
    static constexpr size_t per_warp = (size_t)CAP * (16 * STAGES + 4 + 4 + 2);
};

__device__ __forceinline__ void cmp_swap(uint32_t &a, uint32_t &b)
{
    const uint32_t lo = min(a, b);
    b = max(a, b);
    a = lo;
}

// Sorts E = 2, 4, 8 or 16 words held in registers (Batcher's odd-even merge
// networks: 1, 5, 19 and 63 comparators).
template <int E>
__device__ __forceinline__ void sort_net(uint32_t (&v)[E])
{
    if constexpr (E == 2) {
        cmp_swap(v[0], v[1]);
    } else if constexpr (E == 4) {
        cmp_swap(v[0], v[1]);
        cmp_swap(v[2], v[3]);
        cmp_swap(v[0], v[2]);
        cmp_swap(v[1], v[3]);
        cmp_swap(v[1], v[2]);
    } else if constexpr (E == 16) {
        cmp_swap(v[0], v[1]);
        cmp_swap(v[2], v[3]);
        cmp_swap(v[0], v[2]);
        cmp_swap(v[1], v[3]);
        cmp_swap(v[1], v[2]);
        cmp_swap(v[4], v[5]);
        cmp_swap(v[6], v[7]);
        cmp_swap(v[4], v[6]);
        cmp_swap(v[5], v[7]);
        cmp_swap(v[5], v[6]);
        cmp_swap(v[0], v[4]);
        cmp_swap(v[2], v[6]);
        cmp_swap(v[2], v[4]);
        cmp_swap(v[1], v[5]);
        cmp_swap(v[3], v[7]);
        cmp_swap(v[3], v[5]);
        cmp_swap(v[1], v[2]);
        cmp_swap(v[3], v[4]);
        cmp_swap(v[5], v[6]);
        cmp_swap(v[8], v[9]);
        cmp_swap(v[10], v[11]);
        cmp_swap(v[8], v[10]);
        cmp_swap(v[9], v[11]);
        cmp_swap(v[9], v[10]);
        cmp_swap(v[12], v[13]);
        cmp_swap(v[14], v[15]);
        cmp_swap(v[12], v[14]);
        cmp_swap(v[13], v[15]);
        cmp_swap(v[13], v[14]);
        cmp_swap(v[8], v[12]);
        cmp_swap(v[10], v[14]);
        cmp_swap(v[10], v[12]);
        cmp_swap(v[9], v[13]);
        cmp_swap(v[11], v[15]);
        cmp_swap(v[11], v[13]);
        cmp_swap(v[9], v[10]);
        cmp_swap(v[11], v[12]);
        cmp_swap(v[13], v[14]);
        cmp_swap(v[0], v[8]);
        cmp_swap(v[4], v[12]);
        cmp_swap(v[4], v[8]);
        cmp_swap(v[2], v[10]);
        cmp_swap(v[6], v[14]);
        cmp_swap(v[6], v[10]);
        cmp_swap(v[2], v[4]);
        cmp_swap(v[6], v[8]);
        cmp_swap(v[10], v[12]);
        cmp_swap(v[1], v[9]);
        cmp_swap(v[5], v[13]);
        cmp_swap(v[5], v[9]);
        cmp_swap(v[3], v[11]);
        cmp_swap(v[7], v[15]);
        cmp_swap(v[7], v[11]);
        cmp_swap(v[3], v[5]);
        cmp_swap(v[7], v[9]);
        cmp_swap(v[11], v[13]);
        cmp_swap(v[1], v[2]);
        cmp_swap(v[3], v[4]);
        cmp_swap(v[5], v[6]);
        cmp_swap(v[7], v[8]);
        cmp_swap(v[9], v[10]);
        cmp_swap(v[11], v[12]);
        cmp_swap(v[13], v[14]);
    } else {
        static_assert(E == 8, "sort_net: 2, 4, 8 or 16 words");
        cmp_swap(v[0], v[1]);
        cmp_swap(v[2], v[3]);
        cmp_swap(v[4], v[5]);
        cmp_swap(v[6], v[7]);
        cmp_swap(v[0], v[2]);
        cmp_swap(v[1], v[3]);
        cmp_swap(v[4], v[6]);
        cmp_swap(v[5], v[7]);
        cmp_swap(v[1], v[2]);
        cmp_swap(v[5], v[6]);
        cmp_swap(v[0], v[4]);
        cmp_swap(v[1], v[5]);
        cmp_swap(v[2], v[6]);
        cmp_swap(v[3], v[7]);
        cmp_swap(v[2], v[4]);
        cmp_swap(v[3], v[5]);
        cmp_swap(v[1], v[2]);
        cmp_swap(v[3], v[4]);
        cmp_swap(v[5], v[6]);
    }
}

// Swap rounds of the lane-block sort before the per-element fixup takes
// over (one to three rounds suffice for bucket-ordered random words).
constexpr int kMaxSwapRounds = 32;

// Position, among the n words of one bucket, of the SD of rank rk in full
// (key, rank) order; the keys are drawn again.  Taken only by buckets in
// which two keys share the bits above the rank field (about one cell in 500
// at 256 SDs, one in 60 at 512).
__device__ __noinline__ uint32_t rank_in_bucket_full(uint64_t seed, uint32_t cell, int64_t s, const uint32_t *w,
                                                     uint32_t n, uint32_t rk, uint32_t rank_mask)
{
    auto full_key = [&](uint32_t r) {
        const uint4 k = draw4(seed, r >> 1, cell, s, 0u);
        return (r & 1u) ? (((uint64_t)k.z << 32) | k.w) : (((uint64_t)k.x << 32) | k.y);
    };
    const uint64_t kk = full_key(rk);
    uint32_t c = 0;
    for (uint32_t m = 0; m < n; ++m) {
        const uint32_t r = w[m] & rank_mask;
        c += key_less(full_key(r), r, kk, rk) ? 1u : 0u;
    }
    return c;
}

// FUSED: every cell stays in its stage for n_fused consecutive steps (its
// updates go to the stage, which returns to global memory at the end), for
// runs whose steps have no other dynamic in between; cells are independent,
// so this is the same sequence of steps per cell.  Otherwise one step.  For
// cells up to 256 SDs both forms are bounded to 20 warps per SM (10 blocks
// of 2 warps, 96 registers): the kernel is latency-bound, so more warps beat
// the few spills (the one-step form went from 44.9 to 42.9 us per grid step
// with L2 flushed, the fused form from 30.2 to 27.8).
template <int CAP, int WARPS, int STAGES, bool FUSED = false>
__global__ void __launch_bounds__(32 * WARPS, (CAP <= 256) ? 20 / WARPS : 0) warp_cell_step_kernel(const WorkItem *__restrict__ items, int32_t n_items,
                                                                    InstDev *const *__restrict__ insts,
                                                                    int64_t step_offset, int32_t n_fused = 1)
{
    constexpr int NB = CAP;
    constexpr int LB = ilog2_c(CAP);
    constexpr int RP = CAP / 64 > 0 ? CAP / 64 : 1; // rank pairs per lane
    constexpr int BPL = NB / 32;                   // buckets per lane in the scan
    static_assert((1 << LB) == CAP && CAP >= 64 && CAP <= 512, "warp kernel: CAP in 64..512");
    constexpr unsigned FULL = 0xFFFFFFFFu;
    constexpr int RB = LB > 8 ? LB : 8;      // rank bits of a sort word
    constexpr uint32_t RM = (1u << RB) - 1u; // rank mask
    constexpr int KG = RP < 4 ? RP : 4;      // Philox blocks drawn at a time

    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *mine = smem_raw + (size_t)warp * WarpSmem<CAP, STAGES>::per_warp;
    int64_t *st_xi = reinterpret_cast<int64_t *>(mine);               // [STAGES][CAP]
    double *st_v = reinterpret_cast<double *>(st_xi + STAGES * CAP);  // [STAGES][CAP]
    uint32_t *s_word = reinterpret_cast<uint32_t *>(st_v + STAGES * CAP);
    uint32_t *s_hist = s_word + CAP;
    uint16_t *s_perm = reinterpret_cast<uint16_t *>(s_hist + NB);
    __shared__ uint64_t s_bar_all[WARPS][STAGES];
    __shared__ int4 s_meta_all[WARPS][STAGES];
    uint64_t *s_bar = s_bar_all[warp];
    int4 *s_meta = s_meta_all[warp];

    const int gw = blockIdx.x * WARPS + warp;
    const int nw = gridDim.x * WARPS;
    if (lane == 0) {
        for (int i = 0; i < STAGES; ++i)
            mbar_init(&s_bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    // Lane 0 loads each work item one cell before it issues the item's
    // copies, so that the item's load latency hides behind a cell's work.
    WorkItem nxt{0, 0, 0, 0};
    auto fetch = [&](int k) {
        const int i = gw + k * nw;
        if (i < n_items)
            nxt = items[i];
    };
    auto issue = [&](int k, const WorkItem &it) { // lane 0: start loading this warp's k-th cell
        if (gw + k * nw >= n_items)
            return;
        const int sg = k % STAGES;
        const InstDev *P = insts[it.inst];
        s_meta[sg] = make_int4(it.off, it.n, it.cell, it.inst);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&s_bar[sg], (uint32_t)it.n * 16u);
        bulk_g2s(st_xi + sg * CAP, P->xi + it.off, (uint32_t)it.n * 8u, &s_bar[sg]);
        bulk_g2s(st_v + sg * CAP, P->v + it.off, (uint32_t)it.n * 8u, &s_bar[sg]);
    };

    if (lane == 0) {
        for (int k = 0; k < STAGES - 1; ++k) {
            fetch(k);
            issue(k, nxt);
        }
        fetch(STAGES - 1);
    }

    for (int k = 0; gw + k * nw < n_items; ++k) {
        // Every warp's second cell is asked for only once its first has
        // landed: the first cells of all warps then share the HBM alone at
        // the start of the launch instead of with the second ones.
        const bool defer = STAGES > 1 && k == 0;
        if (lane == 0 && !defer) {
            issue(k + STAGES - 1, nxt);
            fetch(k + STAGES);
        }
        const int sg = k % STAGES;
        const bool arrived = mbar_wait_bounded(&s_bar[sg], (uint32_t)(k / STAGES) & 1u);
        if (!__all_sync(FULL, arrived)) {
            if (lane == 0) {
                atomicOr(&insts[s_meta[sg].w]->status, 1u);
                for (int kk = k; kk < k + (defer ? STAGES - 1 : STAGES); ++kk) // the copies issued
                    if (gw + kk * nw < n_items)
                        mbar_wait_bounded(&s_bar[kk % STAGES], (uint32_t)(kk / STAGES) & 1u);
            }
            return;
        }
        if (lane == 0 && defer) {
            issue(STAGES - 1, nxt);
            fetch(STAGES);
        }
        const int4 meta = s_meta[sg];
        const int n = meta.y;
        const uint32_t cell = (uint32_t)meta.z;
        InstDev *__restrict__ P = insts[meta.w];
        const int64_t s0 = P->step + step_offset;
        const uint64_t seed = P->seed;
        int64_t *xs = st_xi + sg * CAP;
        double *vs = st_v + sg * CAP;
        int64_t *__restrict__ gxi = P->xi + meta.x;
        double *__restrict__ gv = P->v + meta.x;
        // a changed pair goes to global memory, or in FUSED mode to the stage
        auto put_pair = [&](uint32_t a, uint32_t b, int64_t xa, int64_t xb, double va, double vb, bool split) {
            if constexpr (FUSED) {
                xs[a] = xa;
                xs[b] = xb;
                vs[b] = vb;
                if (split)
                    vs[a] = va;
            } else {
                gxi[a] = xa;
                gxi[b] = xb;
                gv[b] = vb;
                if (split)
                    gv[a] = va;
            }
        };
        const int n_rep = FUSED ? n_fused : 1;
        for (int rep = 0; rep < n_rep; ++rep) { // warp-uniform
        const int64_t s = s0 + rep;

        if constexpr (BPL % 4 == 0) {
#pragma unroll
            for (int i = 0; i < BPL / 4; ++i)
                reinterpret_cast<uint4 *>(s_hist)[lane + 32 * i] = make_uint4(0u, 0u, 0u, 0u);
        } else {
#pragma unroll
            for (int i = 0; i < BPL; ++i)
                s_hist[lane + 32 * i] = 0u;
        }
        __syncwarp();

        // Sort words of live SDs and their bucket slots.  A word holds the
        // top 32 - RB bits of the SD's 64-bit key above its RB-bit rank, so
        // words order as (key, rank) except between keys that share those
        // bits; such keys fall in one bucket and the fixup below orders them
        // by their full keys.  Every lane draws KG Philox blocks at a time so
        // that independent chains interleave.
        uint32_t word[2 * RP];
        uint32_t slot[2 * RP];
#pragma unroll
        for (int r0 = 0; r0 < RP; r0 += KG) {
            uint4 kw[KG];
#pragma unroll
            for (int r = 0; r < KG; ++r)
                kw[r] = draw4(seed, (uint32_t)(lane + 32 * (r0 + r)), cell, s, 0u);
#pragma unroll
            for (int r = 0; r < KG; ++r) {
                const int q = lane + 32 * (r0 + r);
                const int i = 2 * (r0 + r);
                slot[i] = 0xFFFFFFFFu;
                slot[i + 1] = 0xFFFFFFFFu;
                word[i] = (kw[r].x & ~RM) | (uint32_t)(2 * q);
                word[i + 1] = (kw[r].z & ~RM) | (uint32_t)(2 * q + 1);
                if (2 * q < n) {
                    const longlong2 x2 = reinterpret_cast<const longlong2 *>(xs)[q];
                    if (x2.x > 0)
                        slot[i] = atomicAdd(&s_hist[word[i] >> (32 - LB)], 1u);
                    if (x2.y > 0)
                        slot[i + 1] = atomicAdd(&s_hist[word[i + 1] >> (32 - LB)], 1u);
                }
            }
        }
        __syncwarp();

        // bucket starts by a warp scan; the total is n_c
        // each lane's BPL buckets are contiguous: read and written as vectors
        // (scalar accesses at this lane stride would conflict 8 ways at 256 SDs)
        uint32_t cnt[BPL], sum = 0;
        if constexpr (BPL % 4 == 0) {
#pragma unroll
            for (int i = 0; i < BPL; i += 4) {
                const uint4 t = reinterpret_cast<const uint4 *>(s_hist + lane * BPL + i)[0];
                cnt[i] = t.x;
                cnt[i + 1] = t.y;
                cnt[i + 2] = t.z;
                cnt[i + 3] = t.w;
            }
        } else if constexpr (BPL == 2) {
            const uint2 t = reinterpret_cast<const uint2 *>(s_hist)[lane];
            cnt[0] = t.x;
            cnt[1] = t.y;
        } else {
#pragma unroll
            for (int i = 0; i < BPL; ++i)
                cnt[i] = s_hist[lane * BPL + i];
        }
#pragma unroll
        for (int i = 0; i < BPL; ++i)
            sum += cnt[i];
        uint32_t incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, d);
            if (lane >= d)
                incl += y;
        }
        const uint32_t n_c = __shfl_sync(FULL, incl, 31);
        uint32_t run = incl - sum;
#pragma unroll
        for (int i = 0; i < BPL; ++i) {
            const uint32_t c = cnt[i];
            cnt[i] = run; // the bucket's start
            run += c;
        }
        if constexpr (BPL % 4 == 0) {
#pragma unroll
            for (int i = 0; i < BPL; i += 4)
                reinterpret_cast<uint4 *>(s_hist + lane * BPL + i)[0] =
                    make_uint4(cnt[i], cnt[i + 1], cnt[i + 2], cnt[i + 3]);
        } else if constexpr (BPL == 2) {
            reinterpret_cast<uint2 *>(s_hist)[lane] = make_uint2(cnt[0], cnt[1]);
        } else {
#pragma unroll
            for (int i = 0; i < BPL; ++i)
                s_hist[lane * BPL + i] = cnt[i];
        }
        __syncwarp();

        if (n_c >= 2) {
#pragma unroll
            for (int i = 0; i < 2 * RP; ++i)
                if (slot[i] != 0xFFFFFFFFu)
                    s_word[s_hist[word[i] >> (32 - LB)] + slot[i]] = word[i];
            __syncwarp();
            // Lane L sorts positions E L .. E L + E - 1 of the bucket-ordered
            // words in registers (positions >= n_c hold 0xFFFFFFFF).  Words
            // can then be out of order only inside buckets that straddle a
            // lane boundary; neighbouring lanes swap inverted boundary words
            // and sort again until no boundary is inverted (every swap
            // removes an inversion).  Equal key prefixes end up adjacent;
            // cells holding one take the per-element fixup with full keys.
            constexpr int E = CAP / 32;
            uint32_t v[E];
            if constexpr (E == 2) {
                const uint2 t = reinterpret_cast<const uint2 *>(s_word)[lane];
                v[0] = t.x;
                v[1] = t.y;
            } else {
#pragma unroll
                for (int i = 0; i < E; i += 4) {
                    const uint4 t = reinterpret_cast<const uint4 *>(s_word + E * lane + i)[0];
                    v[i] = t.x;
                    v[i + 1] = t.y;
                    v[i + 2] = t.z;
                    v[i + 3] = t.w;
                }
            }
#pragma unroll
            for (int i = 0; i < E; ++i)
                if ((uint32_t)(E * lane + i) >= n_c)
                    v[i] = 0xFFFFFFFFu;
            sort_net<E>(v);
            bool fast = true;
            for (int round = 0;; ++round) {
                const uint32_t prev_last = __shfl_up_sync(FULL, v[E - 1], 1);
                const uint32_t next_first = __shfl_down_sync(FULL, v[0], 1);
                const bool lo_inv = lane > 0 && prev_last > v[0];
                const bool hi_inv = lane < 31 && v[E - 1] > next_first;
                if (!__any_sync(FULL, lo_inv || hi_inv))
                    break;
                if (round == kMaxSwapRounds) {
                    fast = false;
                    break;
                }
                if (lo_inv)
                    v[0] = prev_last;
                if (hi_inv)
                    v[E - 1] = next_first;
                sort_net<E>(v);
            }
            // two different words share their key bits iff 1 <= (a ^ b) <= RM
            bool prefix_tie = false;
#pragma unroll
            for (int i = 0; i + 1 < E; ++i)
                prefix_tie |= ((v[i] ^ v[i + 1]) - 1u) < RM;
            const uint32_t nf = __shfl_down_sync(FULL, v[0], 1);
            if (lane < 31)
                prefix_tie |= ((v[E - 1] ^ nf) - 1u) < RM;
            if (fast && !__any_sync(FULL, prefix_tie)) {
                uint32_t pk[E / 2];
#pragma unroll
                for (int i = 0; i < E / 2; ++i)
                    pk[i] = (v[2 * i] & RM) | ((v[2 * i + 1] & RM) << 16);
                if constexpr (E == 2) {
                    reinterpret_cast<uint32_t *>(s_perm)[lane] = pk[0];
                } else if constexpr (E == 4) {
                    reinterpret_cast<uint2 *>(s_perm)[lane] = make_uint2(pk[0], pk[1]);
                } else {
#pragma unroll
                    for (int i = 0; i < E / 8; ++i)
                        reinterpret_cast<uint4 *>(s_perm)[lane * (E / 8) + i] =
                            make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
                }
            } else {
                for (uint32_t pos = lane; pos < n_c; pos += 32) {
                    const uint32_t wv = s_word[pos];
                    const uint32_t b = wv >> (32 - LB);
                    const uint32_t lo = s_hist[b];
                    const uint32_t hi = (b + 1 < (uint32_t)NB) ? s_hist[b + 1] : n_c;
                    uint32_t c = 0;
                    bool tie = false;
                    for (uint32_t m = lo; m < hi; ++m) {
                        const uint32_t wm = s_word[m];
                        c += wm < wv ? 1u : 0u;
                        tie |= ((wm ^ wv) <= RM) & (wm != wv);
                    }
                    if (tie)
                        c = rank_in_bucket_full(seed, cell, s, s_word + lo, hi - lo, wv & RM, RM);
                    s_perm[lo + c] = (uint16_t)(wv & RM);
                }
            }
            __syncwarp();

            // pairs (l = 2q, 2q + 1 share one Philox block).  A bound settles
            // most of them (gamma = 0); the rest are compacted into the sort
            // arrays, dead by now (2 CAP words hold 2 CAP / 3 >= CAP / 2
            // entries of 3 words: every pair fits), and go through the full
            // filter one per lane: certain collisions are updated at once,
            // and so are undecided pairs, after their exact evaluation.
            const uint32_t n_pairs = n_c / 2;
            const float ratio_f = u32_to_f32_rn((n_c & 1u) ? n_c : n_c - 1u);
            const PairConsts C = pair_consts(P);
            const float sc = C.dtdvf * ratio_f;
            const uint32_t n_q = (n_pairs + 1) / 2;
            const uint32_t *vs_words = reinterpret_cast<const uint32_t *>(vs);
            uint32_t *todo = s_word;
            uint32_t n_todo = 0; // warp-uniform
            // QG Philox blocks per lane are drawn, and their pairs bounded,
            // before any compaction, so that the independent chains interleave.
            constexpr int QG = CAP >= 256 ? 2 : 1;
            for (uint32_t q0 = 0; q0 < n_q; q0 += 32 * QG) { // warp-uniform trip count
                uint4 w[QG];
#pragma unroll
                for (int r = 0; r < QG; ++r)
                    w[r] = draw4(seed, q0 + lane + 32 * r, cell, s, 1u);
                bool need[2 * QG];
                uint32_t abv[2 * QG];
#pragma unroll
                for (int r = 0; r < QG; ++r) {
                    const uint32_t q = q0 + lane + 32 * r;
                    uint2 ab2 = make_uint2(0u, 0u); // pairs 2q and 2q + 1
                    if (q < n_q)
                        ab2 = reinterpret_cast<const uint2 *>(s_perm)[q];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t l = 2 * q + h;
                        need[2 * r + h] = false;
                        abv[2 * r + h] = 0;
                        if (q < n_q && l < n_pairs) {
                            // the bound needs xi_j = max(xi_a, xi_b) only; which of the
                            // two is j is settled in the full pass
                            const uint32_t ab = h ? ab2.y : ab2.x;
                            const uint32_t a = ab & 0xFFFFu, b = ab >> 16;
                            const int64_t xa = xs[a], xb = xs[b];
                            abv[2 * r + h] = ab;
                            need[2 * r + h] = !pair_prefilter_zero(C, sc, xa > xb ? xa : xb, vs_words[2 * a + 1],
                                                                   vs_words[2 * b + 1], h ? w[r].z : w[r].x);
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < 2 * QG; ++i) {
                    const unsigned m = __ballot_sync(FULL, need[i]);
                    if (need[i]) {
                        const uint32_t idx = n_todo + __popc(m & ((1u << lane) - 1u));
                        const uint4 &wr = w[i / 2];
                        todo[3 * idx] = abv[i];
                        todo[3 * idx + 1] = (i & 1) ? wr.z : wr.x;
                        todo[3 * idx + 2] = (i & 1) ? wr.w : wr.y;
                    }
                    n_todo += __popc(m);
                }
            }
            __syncwarp();
            for (uint32_t e0 = 0; e0 < n_todo; e0 += 32) { // warp-uniform trip count
                const uint32_t e = e0 + lane;
                uint32_t a = 0, b = 0, wa = 0, wb = 0;
                int32_t gf = 0;
                if (e < n_todo) {
                    const uint32_t ab = todo[3 * e];
                    a = ab & 0xFFFFu;
                    b = ab >> 16;
                    if (xs[a] < xs[b]) { // j holds the larger multiplicity; ties keep the earlier
                        const uint32_t tmp = a;
                        a = b;
                        b = tmp;
                    }
                    wa = todo[3 * e + 1];
                    wb = todo[3 * e + 2];
                    gf = pair_gamma_filter(C, ratio_f, xs[a], vs_words[2 * a + 1], vs_words[2 * b + 1], wa);
                }
                if (gf > 0) { // a certain collision: update from the staged state now
                    int64_t xa = xs[a], xb = xs[b];
                    double va = vs[a], vb = vs[b];
                    const bool split = shima_update(cap_gamma(gf, xa, xb), xa, xb, va, vb);
                    put_pair(a, b, xa, xb, va, vb, split);
                }
                // pairs the filter could not decide: evaluated exactly at
                // once, from the staged copy of the cell
                if (gf < 0) {
                    int64_t xa = xs[a], xb = xs[b];
                    double va = vs[a], vb = vs[b];
                    const int64_t g = pair_gamma_exact(P, n_c, xa, xb, va, vb, wa, wb);
                    if (g > 0) {
                        const bool split = shima_update(g, xa, xb, va, vb);
                        put_pair(a, b, xa, xb, va, vb, split);
                    }
                }
            }
        }
        __syncwarp(); // the work arrays are free again
        } // rep
        if constexpr (FUSED) { // the cell back to global memory
            for (int i = lane; i < n; i += 32) {
                gxi[i] = xs[i];
                gv[i] = vs[i];
            }
            // the stage was written through the generic proxy; the next bulk
            // copy into it goes through the async proxy
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
        }
        // stage sg is free again
    }
}

// ----------------------------------------------------------- big cells
constexpr int kBigChunk = 8192;   // SDs per CTA in the histogram and scatter passes
constexpr int kBigNT = 1024;
constexpr int kBigMaxLB = 14;     // at most 16384 top-level buckets
constexpr int kBucketCap = 1536;  // entries sorted in shared memory per bucket (1024 expected)
constexpr int kBucketNT = 128;
constexpr int kSubLB = 9;         // second-level buckets inside a bucket
constexpr int kPairNT = 128;

struct BigCell {
    int32_t inst, cell;
    int32_t n;        // stored SDs of the cell
    int32_t lb;       // log2 of top-level buckets
    int32_t n_chunks;
    int32_t rcell;    // the cell's index in the random streams (its run's cell_base + cell)
    int64_t hist_base; // into the per-(chunk, bucket) count array
    int64_t sd_base;   // into the key / rank / perm scratch
    int64_t bkt_base;  // into the bucket-start array (2^lb + 1 entries)
};

struct BigChunk {
    int32_t big, chunk;
};
struct BigBucket {
    int32_t big, bucket;
};
struct BigPairs {
    int32_t big, q0; // pair-of-pairs indices q0 .. q0 + kPairNT - 1
};

constexpr int kLiveWords = kBigChunk / 32; // liveness bits of a chunk, in words

struct BigScratch {
    uint32_t *hist;     // per (chunk, bucket) counts, then prefixes
    uint32_t *bstart;   // bucket starts per cell, last entry = n_c
    uint32_t *rank;     // ranks in bucket order (their keys are drawn again where needed)
    uint32_t *perm;     // ranks in sorted order
    double *scale;      // per big cell
    float *scale_f;
    uint32_t *live = nullptr; // kLiveWords per chunk of the launch: which SDs the histogram pass
                              // found live, for the scatter pass (null: the scatter reads xi again)
};

// live SDs of one chunk: keys and their bucket; calls f(key, rank).  Every
// thread of the block calls it.  Liveness comes from xi (live_in null; its
// bits then go to live_out unless that is null too) or from the bits a
// previous call of the same step wrote for the same chunk (live_in): word
// 2 (32 i + warp) + h, bit `lane`, is SD 2q + h of the thread's i-th pair q.
template <typename F>
__device__ __forceinline__ void big_chunk_keys(const InstDev *P, const BigCell &bc, int chunk, int64_t s,
                                               const int64_t *gxi, uint32_t *live_out, const uint32_t *live_in,
                                               F &&f)
{
    constexpr int QPT = kBigChunk / 2 / kBigNT; // SD pairs per thread
    static_assert(QPT * kBigNT * 2 == kBigChunk, "chunk = threads x pairs");
    static_assert(2 * QPT * (kBigNT / 32) == kLiveWords, "a chunk's liveness words");
    const int lo2 = (chunk * kBigChunk) / 2;
    const int hi2 = min((chunk + 1) * kBigChunk, bc.n) / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool lx[QPT], ly[QPT];
    if (live_in) {
        uint2 m[QPT];
#pragma unroll
        for (int i = 0; i < QPT; ++i)
            m[i] = reinterpret_cast<const uint2 *>(live_in)[i * (kBigNT / 32) + warp];
#pragma unroll
        for (int i = 0; i < QPT; ++i) {
            lx[i] = (m[i].x >> lane) & 1u;
            ly[i] = (m[i].y >> lane) & 1u;
        }
    } else {
        // every load of the thread first, so that they are in flight together
        longlong2 x[QPT];
#pragma unroll
        for (int i = 0; i < QPT; ++i) {
            const int q = lo2 + (int)threadIdx.x + i * kBigNT;
            x[i] = q < hi2 ? reinterpret_cast<const longlong2 *>(gxi)[q] : make_longlong2(0, 0);
        }
#pragma unroll
        for (int i = 0; i < QPT; ++i) {
            lx[i] = x[i].x > 0;
            ly[i] = x[i].y > 0;
        }
        if (live_out) {
#pragma unroll
            for (int i = 0; i < QPT; ++i) {
                const unsigned bx = __ballot_sync(0xFFFFFFFFu, lx[i]), by = __ballot_sync(0xFFFFFFFFu, ly[i]);
                if (lane == 0)
                    reinterpret_cast<uint2 *>(live_out)[i * (kBigNT / 32) + warp] = make_uint2(bx, by);
            }
        }
    }
    const uint64_t seed = P->seed;
#pragma unroll
    for (int i = 0; i < QPT; ++i) {
        const int q = lo2 + (int)threadIdx.x + i * kBigNT;
        if (lx[i] | ly[i]) {
            const uint4 w = draw4(seed, (uint32_t)q, (uint32_t)bc.rcell, s, 0u);
            if (lx[i])
                f(((uint64_t)w.x << 32) | w.y, (uint32_t)(2 * q));
            if (ly[i])
                f(((uint64_t)w.z << 32) | w.w, (uint32_t)(2 * q + 1));
        }
    }
}

__global__ void __launch_bounds__(kBigNT) big_hist_kernel(const BigChunk *__restrict__ chunks,
                                                          const BigCell *__restrict__ bigs,
                                                          const InstDev *const *__restrict__ insts,
                                                          BigScratch S, int64_t step_offset)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem_raw);
    const BigChunk ch = chunks[blockIdx.x];
    const BigCell bc = bigs[ch.big];
    const InstDev *P = insts[bc.inst];
    const int NB = 1 << bc.lb;
    for (int i = threadIdx.x; i < NB; i += kBigNT)
        s_hist[i] = 0u;
    __syncthreads();
    const int64_t s = P->step + step_offset;
    const int64_t *gxi = P->xi + P->cell_off[bc.cell];
    const int sh = 64 - bc.lb;
    uint32_t *live = S.live ? S.live + (size_t)blockIdx.x * kLiveWords : nullptr;
    big_chunk_keys(P, bc, ch.chunk, s, gxi, live, nullptr,
                   [&](uint64_t k, uint32_t) { atomicAdd(&s_hist[k >> sh], 1u); });
    __syncthreads();
    uint32_t *h = S.hist + bc.hist_base + (int64_t)ch.chunk * NB;
    for (int i = threadIdx.x; i < NB; i += kBigNT)
        h[i] = s_hist[i];
}

// Per bucket of a big cell, the running prefix of its counts over the chunks
// (in place) and the bucket total (into the bucket-start array, scanned
// next).  Block (big, tile) takes buckets 256 tile .. 256 tile + 255 of big
// cell `big`; each thread loads its column kBigColU chunks at a time.
constexpr int kBigColNT = 256;
constexpr int kBigColU = 16;

__global__ void __launch_bounds__(kBigColNT) big_colscan_kernel(const BigCell *__restrict__ bigs, int32_t max_tiles,
                                                                BigScratch S)
{
    const int big = blockIdx.x / max_tiles, tile = blockIdx.x - big * max_tiles;
    const BigCell bc = bigs[big];
    const int NB = 1 << bc.lb;
    const int b = tile * kBigColNT + threadIdx.x;
    if (b >= NB)
        return;
    uint32_t *h = S.hist + bc.hist_base;
    uint32_t run = 0;
    for (int c0 = 0; c0 < bc.n_chunks; c0 += kBigColU) {
        uint32_t x[kBigColU];
#pragma unroll
        for (int u = 0; u < kBigColU; ++u)
            x[u] = c0 + u < bc.n_chunks ? h[(int64_t)(c0 + u) * NB + b] : 0u;
#pragma unroll
        for (int u = 0; u < kBigColU; ++u) {
            if (c0 + u < bc.n_chunks)
                h[(int64_t)(c0 + u) * NB + b] = run;
            run += x[u];
        }
    }
    S.bstart[bc.bkt_base + b] = run;
}

// One CTA per big cell: bucket starts from the bucket totals; the cell's
// scale factor.
__global__ void __launch_bounds__(kBigNT) big_scan_kernel(const BigCell *__restrict__ bigs,
                                                          const InstDev *const *__restrict__ insts, BigScratch S)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint32_t *s_tot = reinterpret_cast<uint32_t *>(smem_raw);
    __shared__ uint32_t s_warp[32];
    const BigCell bc = bigs[blockIdx.x];
    const int NB = 1 << bc.lb;
    for (int b = threadIdx.x; b < NB; b += kBigNT)
        s_tot[b] = S.bstart[bc.bkt_base + b];
    for (int b = NB + threadIdx.x; b < (1 << kBigMaxLB); b += kBigNT)
        s_tot[b] = 0u;
    __syncthreads();
    const uint32_t n_c = block_exclusive_scan<kBigNT, (1 << kBigMaxLB)>(s_tot, s_warp);
    uint32_t *bs = S.bstart + bc.bkt_base;
    for (int b = threadIdx.x; b < NB; b += kBigNT)
        bs[b] = s_tot[b];
    if (threadIdx.x == 0) {
        bs[NB] = n_c;
        const double sc = n_c >= 2 ? cell_scale(insts[bc.inst]->dtdv, (int64_t)n_c) : 0.0;
        S.scale[blockIdx.x] = sc;
        S.scale_f[blockIdx.x] = __double2float_rn(sc);
    }
}

__global__ void __launch_bounds__(kBigNT) big_scatter_kernel(const BigChunk *__restrict__ chunks,
                                                             const BigCell *__restrict__ bigs,
                                                             const InstDev *const *__restrict__ insts,
                                                             BigScratch S, int64_t step_offset)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint32_t *s_cnt = reinterpret_cast<uint32_t *>(smem_raw);
    const BigChunk ch = chunks[blockIdx.x];
    const BigCell bc = bigs[ch.big];
    const InstDev *P = insts[bc.inst];
    const int NB = 1 << bc.lb;
    // this chunk's first slot in every bucket
    const uint32_t *h = S.hist + bc.hist_base + (int64_t)ch.chunk * NB;
    const uint32_t *bs = S.bstart + bc.bkt_base;
    for (int i = threadIdx.x; i < NB; i += kBigNT)
        s_cnt[i] = bs[i] + h[i];
    __syncthreads();
    const int64_t s = P->step + step_offset;
    const int64_t *gxi = P->xi + P->cell_off[bc.cell];
    const int sh = 64 - bc.lb;
    uint32_t *rout = S.rank + bc.sd_base;
    // only the rank is stored (4 bytes, not 12 with the key): the scattered
    // writes then stay in L2 instead of costing partial-sector rewrites
    // liveness as the histogram pass of this step found it (same chunk
    // list and grid), so xi is not read again
    const uint32_t *live = S.live ? S.live + (size_t)blockIdx.x * kLiveWords : nullptr;
    big_chunk_keys(P, bc, ch.chunk, s, gxi, nullptr, live, [&](uint64_t k, uint32_t rank) {
        rout[atomicAdd(&s_cnt[(uint32_t)(k >> sh)], 1u)] = rank;
    });
}

// The 64-bit sort key of the SD of rank r in a big cell (as big_chunk_keys).
__device__ __forceinline__ uint64_t big_key(uint64_t seed, uint32_t cell, int64_t s, uint32_t r)
{
    const uint4 w = draw4(seed, r >> 1, cell, s, 0u);
    return (r & 1u) ? (((uint64_t)w.z << 32) | w.w) : (((uint64_t)w.x << 32) | w.y);
}

// One CTA per top-level bucket: draw its entries' keys again, order them by
// (key, rank) through second-level buckets on the next kSubLB key bits,
// write the ranks to perm.
__global__ void __launch_bounds__(kBucketNT) big_bucket_sort_kernel(const BigBucket *__restrict__ work,
                                                                    const BigCell *__restrict__ bigs,
                                                                    const InstDev *const *__restrict__ insts,
                                                                    BigScratch S, int64_t step_offset)
{
    constexpr int NSB = 1 << kSubLB;
    constexpr int R = kBucketCap / kBucketNT;
    __shared__ uint32_t s_hist[NSB];
    __shared__ uint64_t s_key[kBucketCap];
    __shared__ uint32_t s_rank[kBucketCap];
    __shared__ uint32_t s_warp[32];
    const BigBucket bw = work[blockIdx.x];
    const BigCell bc = bigs[bw.big];
    const uint32_t *bs = S.bstart + bc.bkt_base;
    const uint32_t lo = bs[bw.bucket], hi = bs[bw.bucket + 1];
    const uint32_t nb = hi - lo;
    const uint32_t *rin = S.rank + bc.sd_base + lo;
    uint32_t *pout = S.perm + bc.sd_base + lo;
    if (nb == 0)
        return;
    const InstDev *P = insts[bc.inst];
    const uint64_t seed = P->seed;
    const int64_t s = P->step + step_offset;
    const uint32_t cell = (uint32_t)bc.rcell;
    if (nb > (uint32_t)kBucketCap) {
        // overfull bucket (never expected for uniform keys): rank by counting
        for (uint32_t e = threadIdx.x; e < nb; e += kBucketNT) {
            const uint32_t r = rin[e];
            const uint64_t k = big_key(seed, cell, s, r);
            uint32_t cnt = 0;
            for (uint32_t m = 0; m < nb; ++m)
                cnt += key_less(big_key(seed, cell, s, rin[m]), rin[m], k, r) ? 1u : 0u;
            pout[cnt] = r;
        }
        return;
    }
    for (int i = threadIdx.x; i < NSB; i += kBucketNT)
        s_hist[i] = 0u;
    __syncthreads();
    const int sh = 64 - bc.lb - kSubLB;
    uint64_t key[R];
    uint32_t rank[R], slot[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t e = threadIdx.x + r * kBucketNT;
        slot[r] = 0xFFFFFFFFu;
        if (e < nb) {
            rank[r] = rin[e];
            key[r] = big_key(seed, cell, s, rank[r]);
            slot[r] = atomicAdd(&s_hist[(key[r] >> sh) & (NSB - 1)], 1u);
        }
    }
    __syncthreads();
    block_exclusive_scan<kBucketNT, NSB>(s_hist, s_warp);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (slot[r] != 0xFFFFFFFFu) {
            const uint32_t pos = s_hist[(key[r] >> sh) & (NSB - 1)] + slot[r];
            s_key[pos] = key[r];
            s_rank[pos] = rank[r];
        }
    }
    __syncthreads();
    for (uint32_t pos = threadIdx.x; pos < nb; pos += kBucketNT) {
        const uint64_t k = s_key[pos];
        const uint32_t rk = s_rank[pos];
        const uint32_t b = (uint32_t)((k >> sh) & (NSB - 1));
        const uint32_t blo = s_hist[b];
        const uint32_t bhi = (b + 1 < (uint32_t)NSB) ? s_hist[b + 1] : nb;
        uint32_t cnt = 0;
        for (uint32_t m = blo; m < bhi; ++m)
            cnt += key_less(s_key[m], s_rank[m], k, rk) ? 1u : 0u;
        pout[blo + cnt] = rk;
    }
}

__global__ void __launch_bounds__(kPairNT) big_pairs_kernel(const BigPairs *__restrict__ work,
                                                            const BigCell *__restrict__ bigs,
                                                            InstDev *const *__restrict__ insts,
                                                            BigScratch S, int64_t step_offset)
{
    const BigPairs pw = work[blockIdx.x];
    const int big = pw.big;
    const BigCell bc = bigs[big];
    const uint32_t n_c = S.bstart[bc.bkt_base + (1 << bc.lb)];
    const uint32_t n_pairs = n_c / 2;
    const uint32_t q = (uint32_t)pw.q0 + threadIdx.x;
    if (2 * q >= n_pairs)
        return;
    const InstDev *__restrict__ P = insts[bc.inst];
    const PairConsts C = pair_consts(P);
    const int64_t s = P->step + step_offset;
    const int32_t off = P->cell_off[bc.cell];
    int64_t *__restrict__ gxi = P->xi + off;
    double *__restrict__ gv = P->v + off;
    const uint32_t *perm = S.perm + bc.sd_base;
    const float ratio_f = u32_to_f32_rn((n_c & 1u) ? n_c : n_c - 1u);
    const uint4 w = draw4(P->seed, q, (uint32_t)bc.rcell, s, 1u);
    // both pairs' SDs are gathered at once (eight independent loads)
    uint32_t A[2], B[2];
    int64_t XA[2], XB[2];
    double VA[2], VB[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t l = 2 * q + h;
        A[h] = B[h] = 0;
        if (l < n_pairs) {
            const uint2 ab = reinterpret_cast<const uint2 *>(perm)[l];
            A[h] = ab.x;
            B[h] = ab.y;
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        XA[h] = XB[h] = 0;
        VA[h] = VB[h] = 0.0;
        if (2 * q + h < n_pairs) {
            XA[h] = gxi[A[h]];
            XB[h] = gxi[B[h]];
            VA[h] = gv[A[h]];
            VB[h] = gv[B[h]];
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t l = 2 * q + h;
        if (l >= n_pairs)
            break;
        uint32_t a = A[h], b = B[h];
        int64_t xa = XA[h], xb = XB[h];
        double va = VA[h], vb = VB[h];
        if (xa < xb) { // j holds the larger multiplicity; ties keep the earlier
            const uint32_t tmp = a;
            a = b;
            b = tmp;
            const int64_t tx = xa;
            xa = xb;
            xb = tx;
            const double tv = va;
            va = vb;
            vb = tv;
        }
        const uint32_t wa = h ? w.z : w.x, wb = h ? w.w : w.y;
        const int32_t gf = pair_gamma_filter(C, ratio_f, xa, va, vb, wa);
        if (gf == 0)
            continue;
        const int64_t g = gf > 0 ? cap_gamma(gf, xa, xb) : pair_gamma_exact(P, n_c, xa, xb, va, vb, wa, wb);
        if (g > 0) {
            const bool split = shima_update(g, xa, xb, va, vb);
            gxi[a] = xa;
            gxi[b] = xb;
            gv[b] = vb;
            if (split)
                gv[a] = va;
        }
    }
}

// Step counters.  Kernels read base + step_offset, where step_offset is a
// launch argument; the device base only moves here: by n for every run (the
// tail of a captured graph), or by a per-run delta (delta != nullptr).
__global__ void advance_steps_kernel(InstDev *const *insts, int32_t n_inst, int64_t n, const int64_t *delta)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_inst)
        insts[i]->step += delta ? delta[i] : n;
}

// ------------------------------------------------------------ diagnostics
// Conservation sums of the SDs inside the domain (slots [0, n_in)): live
// count, sum of xi (128-bit, exact) and sum of xi v (binary64).  Each thread
// adds its slots in index order, then warps and blocks combine in a fixed
// tree, so that a given grid gives the same bits every time.
struct DiagPart {
    unsigned long long live, xi_lo, xi_hi;
    double xv;
};
constexpr int kDiagNT = 256;

__device__ __forceinline__ void add128(unsigned long long &lo, unsigned long long &hi, unsigned long long blo,
                                       unsigned long long bhi)
{
    const unsigned long long s = lo + blo;
    hi += bhi + (s < lo ? 1ull : 0ull);
    lo = s;
}

__device__ __forceinline__ void diag_combine(DiagPart &a, const DiagPart &b)
{
    a.live += b.live;
    add128(a.xi_lo, a.xi_hi, b.xi_lo, b.xi_hi);
    a.xv = __dadd_rn(a.xv, b.xv);
}

__device__ __forceinline__ DiagPart diag_shfl_down(const DiagPart &a, int d)
{
    DiagPart b;
    b.live = __shfl_down_sync(0xFFFFFFFFu, a.live, d);
    b.xi_lo = __shfl_down_sync(0xFFFFFFFFu, a.xi_lo, d);
    b.xi_hi = __shfl_down_sync(0xFFFFFFFFu, a.xi_hi, d);
    b.xv = __shfl_down_sync(0xFFFFFFFFu, a.xv, d);
    return b;
}

// fixed tree over the block: lanes within warps, then warps (thread 0 ends with the block's sum)
__device__ __forceinline__ DiagPart diag_block_reduce(DiagPart a)
{
    __shared__ DiagPart s_w[kDiagNT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const DiagPart b = diag_shfl_down(a, d);
        diag_combine(a, b);
    }
    if (lane == 0)
        s_w[warp] = a;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < kDiagNT / 32; ++w)
            diag_combine(a, s_w[w]);
    return a;
}

__global__ void __launch_bounds__(kDiagNT) diag_partial_kernel(const InstDev *__restrict__ P, int64_t n_in,
                                                               DiagPart *__restrict__ parts)
{
    DiagPart a{0ull, 0ull, 0ull, 0.0};
    const int64_t stride = (int64_t)gridDim.x * kDiagNT;
    for (int64_t i = (int64_t)blockIdx.x * kDiagNT + threadIdx.x; i < n_in; i += stride) {
        const int64_t x = P->xi[i];
        if (x > 0) {
            a.live += 1ull;
            add128(a.xi_lo, a.xi_hi, (unsigned long long)x, 0ull);
            a.xv = __fma_rn(xi2d(x), P->v[i], a.xv);
        }
    }
    a = diag_block_reduce(a);
    if (threadIdx.x == 0)
        parts[blockIdx.x] = a;
}

__global__ void __launch_bounds__(kDiagNT) diag_final_kernel(const DiagPart *__restrict__ parts, int32_t n_parts,
                                                             DiagPart *__restrict__ out)
{
    DiagPart a{0ull, 0ull, 0ull, 0.0};
    for (int i = threadIdx.x; i < n_parts; i += kDiagNT)
        diag_combine(a, parts[i]);
    a = diag_block_reduce(a);
    if (threadIdx.x == 0)
        *out = a;
}

// -------------------------------------------------------------- spectrum
constexpr int kSpecNT = 256;
constexpr int kMaxEdges = 1024;

// Bin of a live SD of volume v among the edges (-1: outside [e_0, e_N)).
// The binary32 radius decides when it lies clear (2^-14 relative) of every
// bin edge, else the exact binary64 radius and search do.
__device__ __forceinline__ int spectrum_bin(double v, const double *s_edges, const float *s_lo, const float *s_hi,
                                            int n_edges)
{
    const int nb = n_edges - 1;
    bool in_range;
    const float rf = cbrt_filter(hi2f((uint32_t)__double2hiint(v), in_range) * kVolToR3F);
    // largest lo with lower(edge[lo]) <= rf
    int lo = -1, hi = n_edges;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_lo[mid] <= rf)
            lo = mid;
        else
            hi = mid;
    }
    const bool clear_below = lo >= 0 && rf > s_hi[lo];
    const bool clear_above = lo + 1 >= n_edges || rf < s_lo[lo + 1];
    if (in_range && (lo < 0 || clear_below) && clear_above)
        return (lo < 0 || lo >= nb) ? -1 : lo;
    const double r = radius_exact(v);
    if (r < s_edges[0] || !(r < s_edges[n_edges - 1]))
        return -1;
    int a = 0, z = n_edges - 1;
    while (z - a > 1) {
        const int mid = (a + z) >> 1;
        if (s_edges[mid] <= r)
            a = mid;
        else
            z = mid;
    }
    return a;
}

// The same with a fixed-step search over at most MAXE - 1 edges (unrolled,
// so that the searches of neighbouring SDs interleave).
template <int MAXE>
__device__ __forceinline__ int spectrum_bin_fixed(double v, const double *s_edges, const float *s_lo,
                                                  const float *s_hi, int n_edges)
{
    const int nb = n_edges - 1;
    bool in_range;
    const float rf = cbrt_filter(hi2f((uint32_t)__double2hiint(v), in_range) * kVolToR3F);
    int lo = -1; // largest lo with lower(edge[lo]) <= rf
#pragma unroll
    for (int step = MAXE / 2; step > 0; step >>= 1) {
        const int mid = lo + step;
        if (mid < n_edges && s_lo[mid] <= rf)
            lo = mid;
    }
    const bool clear_below = lo >= 0 && rf > s_hi[lo];
    const bool clear_above = lo + 1 >= n_edges || rf < s_lo[lo + 1];
    if (in_range && (lo < 0 || clear_below) && clear_above)
        return (lo < 0 || lo >= nb) ? -1 : lo;
    return spectrum_bin(v, s_edges, s_lo, s_hi, n_edges);
}

// Edges into shared memory with their binary32 images widened by 2^-14.
__device__ __forceinline__ void spectrum_edges_to_smem(const double *edges, int n_edges, double *s_edges, float *s_lo,
                                                       float *s_hi)
{
    for (int i = threadIdx.x; i < n_edges; i += blockDim.x) {
        const double e = edges[i];
        s_edges[i] = e;
        const float ef = __double2float_rn(e);
        s_lo[i] = ef * (1.0f - 0x1p-14f);
        s_hi[i] = ef * (1.0f + 0x1p-14f);
    }
}

// dv/dlnr accumulation, one block per cell: sum of xi v per bin of live SDs.
// per_cell: acc[cell * nb + b]; otherwise atomically into acc[b].
__global__ void __launch_bounds__(kSpecNT) spectrum_kernel(const InstDev *__restrict__ P, const double *__restrict__ edges,
                                                           int32_t n_edges, int32_t per_cell, double *__restrict__ acc)
{
    __shared__ double s_edges[kMaxEdges];
    __shared__ float s_lo[kMaxEdges], s_hi[kMaxEdges]; // edges widened by 2^-14 either way
    __shared__ double s_acc[kMaxEdges];
    const int cell = blockIdx.x;
    const int nb = n_edges - 1;
    spectrum_edges_to_smem(edges, n_edges, s_edges, s_lo, s_hi);
    for (int i = threadIdx.x; i < nb; i += kSpecNT)
        s_acc[i] = 0.0;
    __syncthreads();
    const int32_t off = P->cell_off[cell];
    const int n = P->cell_off[cell + 1] - off;
    const int64_t *gxi = P->xi + off;
    const double *gv = P->v + off;
    for (int i = threadIdx.x; i < n; i += kSpecNT) {
        const int64_t x = gxi[i];
        if (x <= 0)
            continue;
        const double v = gv[i];
        const int bin = spectrum_bin(v, s_edges, s_lo, s_hi, n_edges);
        if (bin >= 0)
            atomicAdd(&s_acc[bin], __dmul_rn(xi2d(x), v));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += kSpecNT) {
        if (per_cell)
            acc[(int64_t)cell * nb + b] = s_acc[b];
        else if (s_acc[b] != 0.0)
            atomicAdd(&acc[b], s_acc[b]);
    }
}

// Total spectrum without atomics: a grid-stride pass over every storage slot
// (padding and dead SDs hold xi = 0); each thread adds into its own column
// of a bins x threads shared array, then each block sums its columns in a
// fixed order into partial[bin][block].  Results repeat bit for bit.
constexpr int kSpecTotNT = 128;
constexpr int kSpecTotMaxBins = 32;

__global__ void __launch_bounds__(kSpecTotNT) spectrum_total_kernel(const InstDev *__restrict__ P, int64_t n_slots,
                                                                    const double *__restrict__ edges, int32_t n_edges,
                                                                    double *__restrict__ partial)
{
    __shared__ double s_col[kSpecTotMaxBins * kSpecTotNT];
    __shared__ double s_edges[kSpecTotMaxBins + 1];
    __shared__ float s_lo[kSpecTotMaxBins + 1], s_hi[kSpecTotMaxBins + 1];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nb = n_edges - 1;
    spectrum_edges_to_smem(edges, n_edges, s_edges, s_lo, s_hi);
    for (int b = 0; b < nb; ++b)
        s_col[b * kSpecTotNT + t] = 0.0;
    __syncthreads();
    const int64_t *__restrict__ gxi = P->xi;
    const double *__restrict__ gv = P->v;
    // four slots per iteration, all loads issued before any is used
    constexpr int U = 4;
    const int64_t stride = (int64_t)gridDim.x * kSpecTotNT;
    for (int64_t i0 = (int64_t)blockIdx.x * kSpecTotNT + t; i0 < n_slots; i0 += U * stride) {
        int64_t x[U];
        double v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = i0 + u * stride;
            x[u] = i < n_slots ? gxi[i] : 0;
            v[u] = i < n_slots ? gv[i] : 1.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (x[u] <= 0)
                continue;
            const int bin = spectrum_bin_fixed<2 * kSpecTotMaxBins>(v[u], s_edges, s_lo, s_hi, n_edges);
            if (bin >= 0) // xi v added with one rounding
                s_col[bin * kSpecTotNT + t] = __fma_rn(xi2d(x[u]), v[u], s_col[bin * kSpecTotNT + t]);
        }
    }
    __syncthreads();
    // Bins that no thread of the block touched hold zeros only: they skip the
    // binary64 adds (adding +0.0 changes no sum, so the result is the same).
    for (int b = warp; b < nb; b += kSpecTotNT / 32) {
        bool any = false;
        for (int j = lane; j < kSpecTotNT; j += 32)
            any |= s_col[b * kSpecTotNT + j] != 0.0;
        double sum = 0.0;
        if (__any_sync(0xFFFFFFFFu, any)) {
            for (int j = lane; j < kSpecTotNT; j += 32)
                sum = __dadd_rn(sum, s_col[b * kSpecTotNT + j]);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1)
                sum = __dadd_rn(sum, __shfl_down_sync(0xFFFFFFFFu, sum, d));
        }
        if (lane == 0)
            partial[(int64_t)b * gridDim.x + blockIdx.x] = sum;
    }
}

// out[b] = (sum over blocks of partial[b][block], fixed order) / vol / dln[b],
// dln[b] = ln e[b+1] - ln e[b] (from the host); one warp (block) per bin.
__global__ void spectrum_total_finalize_kernel(const double *__restrict__ partial, int32_t n_blocks,
                                               const double *__restrict__ dln, int32_t nb, double vol,
                                               double *__restrict__ out)
{
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31;
    if (b >= nb)
        return;
    double sum = 0.0;
    for (int j = lane; j < n_blocks; j += 32)
        sum = __dadd_rn(sum, partial[(int64_t)b * n_blocks + j]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
        sum = __dadd_rn(sum, __shfl_down_sync(0xFFFFFFFFu, sum, d));
    if (lane == 0)
        out[b] = sum / vol / dln[b];
}

// out[i] = acc[i] / vol / dln[i mod nb]
__global__ void spectrum_finalize_kernel(const double *__restrict__ acc, const double *__restrict__ dln, int32_t nb,
                                         int64_t n_out, double vol, double *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_out)
        return;
    out[i] = acc[i] / vol / dln[i % nb];
}

// --------------------------------------------------------------- layout
// Validation and per-group counts of set_attributes (groups: the cells, then
// n_cells for the SDs outside the domain, cell id -1).  flags bit 0: an
// invalid attribute (first bad SD index in *bad); bit 1: groups not sorted.
// Each warp takes 32 consecutive SDs at a time and adds one count per run of
// equal groups (one or two atomics per warp for sorted input).
__global__ void validate_count_kernel(int64_t lo, int64_t hi, const int64_t *__restrict__ xi,
                                      const double *__restrict__ v, const int32_t *__restrict__ cell, int32_t n_cells,
                                      uint32_t *__restrict__ counts, uint32_t *__restrict__ flags,
                                      unsigned long long *__restrict__ bad)
{
    constexpr unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = lo + (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < hi; base += wstride) {
        const int64_t i = base + lane;
        const bool in = i < hi;
        const int32_t c_in = in ? cell[i] : INT32_MAX;
        const int32_t craw = c_in == -1 ? n_cells : c_in; // the group; outside sorts last
        int32_t c = -1;                                     // counted group, -1: none
        if (in) {
            const double vi = v[i];
            if (xi[i] >= 0 && vi >= 1e-30 && vi <= 1e30 && c_in >= -1 && c_in < n_cells) {
                c = craw;
            } else {
                atomicOr(flags, 1u);
                atomicMin(bad, (unsigned long long)i);
            }
        }
        int32_t prev = __shfl_up_sync(FULL, craw, 1);
        if (lane == 0) {
            prev = INT32_MIN;
            if (in && i > 0)
                prev = cell[i - 1] == -1 ? n_cells : cell[i - 1];
        }
        if (__any_sync(FULL, in && prev > craw) && lane == 0)
            atomicOr(flags, 2u);
        const int32_t next = __shfl_down_sync(FULL, c, 1);
        const bool end = lane == 31 || next != c;
        const unsigned ends = __ballot_sync(FULL, end);
        if (end && c >= 0) {
            const unsigned below = ends & ((1u << lane) - 1u);
            const int start = below ? 32 - __clz(below) : 0;
            atomicAdd(&counts[c], (uint32_t)(lane - start + 1));
        }
    }
}

// Group-sorted input: SD i goes to padded slot poff[g] + (i - uoff[g]), g its
// group (cell id -1: n_cells, outside the domain).  Otherwise pos[i] gives
// the slot.
__global__ void scatter_kernel(int64_t n_sd, const int64_t *__restrict__ xi, const double *__restrict__ v,
                               const int32_t *__restrict__ cell, int32_t n_cells, const int32_t *__restrict__ poff,
                               const int32_t *__restrict__ uoff, const int32_t *__restrict__ pos,
                               int64_t *__restrict__ sxi, double *__restrict__ sv, int32_t *__restrict__ id_of_slot)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_sd; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t p;
        if (pos) {
            p = pos[i];
        } else {
            const int32_t c = cell[i] < 0 ? n_cells : cell[i];
            p = poff[c] + (int32_t)(i - uoff[c]);
        }
        sxi[p] = xi[i];
        sv[p] = v[i];
        id_of_slot[p] = (int32_t)i;
    }
}

// Padding slots (the one slot after an odd group): dead, with a harmless
// positive volume.
__global__ void fill_padding_kernel(int32_t n_cells, const int32_t *__restrict__ poff, const int32_t *__restrict__ uoff,
                                    int64_t *__restrict__ sxi, double *__restrict__ sv, int32_t *__restrict__ id_of_slot)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x) {
        for (int32_t p = poff[c] + (uoff[c + 1] - uoff[c]); p < poff[c + 1]; ++p) {
            sxi[p] = 0;
            sv[p] = 1.0;
            id_of_slot[p] = -1;
        }
    }
}

__global__ void gather_kernel(int64_t n_slots, const int64_t *__restrict__ sxi, const double *__restrict__ sv,
                              const int32_t *__restrict__ id_of_slot, int64_t *__restrict__ xi, double *__restrict__ v)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_slots; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t id = id_of_slot[p];
        if (id < 0)
            continue;
        if (xi)
            xi[id] = sxi[p];
        if (v)
            v[id] = sv[p];
    }
}

} // namespace sdm
