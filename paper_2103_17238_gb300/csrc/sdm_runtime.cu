// C-ABI runtime of the SDM coalescence library: contexts, attribute layout,
// batch plans (work lists per cell-size class, big-cell scratch), launches,
// CUDA-graph replay, the spectrum product.  Declarations and the contract of
// every call are in include/sdm.h.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sdm.h"
#include "sdm_kernels.cuh"
#include "sdm_mid.cuh"

using namespace sdm;

namespace {

thread_local std::string g_thread_error;

// An NVTX range around each C-ABI call (a profiler's timeline shows the
// calls; without an attached tool a push or pop costs a few nanoseconds).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct DevMem {
    sdm_alloc_fn fn = nullptr;
    sdm_free_fn ffn = nullptr;
    void *user = nullptr;
    cudaStream_t stream = nullptr;
    // Small blocks (per-call scratch: validation counts, offsets, spectrum
    // partials) are kept for the next call instead of going back through the
    // allocator hook each time.  Every use is ordered on this stream, so a
    // block handed out again follows its last use.
    static constexpr size_t kKeepMax = (size_t)1 << 19; // bytes
    static constexpr size_t kKeepBlocks = 6;
    struct Block {
        void *p;
        size_t bytes;
    };
    std::vector<Block> kept; // free blocks
    std::vector<Block> lent; // kept-size blocks in use (their true sizes)

    void *raw_get(size_t bytes)
    {
        if (fn)
            return fn(bytes, (void *)stream, user);
        void *p = nullptr;
        if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void raw_put(void *p, size_t bytes)
    {
        if (ffn)
            ffn(p, bytes, (void *)stream, user);
        else
            cudaFreeAsync(p, stream);
    }
    void *get(size_t bytes)
    {
        if (bytes == 0)
            bytes = 16;
        if (bytes > kKeepMax)
            return raw_get(bytes);
        size_t best = kept.size();
        for (size_t i = 0; i < kept.size(); ++i)
            if (kept[i].bytes >= bytes && (best == kept.size() || kept[i].bytes < kept[best].bytes))
                best = i;
        Block b;
        if (best < kept.size()) {
            b = kept[best];
            kept.erase(kept.begin() + (std::ptrdiff_t)best);
        } else {
            b.bytes = bytes;
            b.p = raw_get(bytes);
            if (!b.p)
                return nullptr;
        }
        lent.push_back(b);
        return b.p;
    }
    void put(void *p, size_t bytes)
    {
        if (!p)
            return;
        for (size_t i = 0; i < lent.size(); ++i)
            if (lent[i].p == p) {
                const Block b = lent[i];
                lent.erase(lent.begin() + (std::ptrdiff_t)i);
                if (kept.size() < kKeepBlocks)
                    kept.push_back(b);
                else
                    raw_put(b.p, b.bytes);
                return;
            }
        raw_put(p, bytes);
    }
    DevMem() = default;
    // The block lists belong to one owner: a second owner takes the hooks only.
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
    void use_hooks_of(const DevMem &o, cudaStream_t s)
    {
        fn = o.fn;
        ffn = o.ffn;
        user = o.user;
        stream = s;
    }
    // returns the kept blocks to the allocator (before the owner goes away)
    void release_kept()
    {
        for (const Block &b : kept)
            raw_put(b.p, b.bytes);
        kept.clear();
    }
};

// A device buffer owned through DevMem.
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

constexpr int kInChunks = 4; // pieces of a host input copy (sdm_set_attributes)

// Cell-size classes of the shared-memory path.
constexpr int kClassCap[] = {64, 128, 256, 512, 1024, 2048, 4096};
constexpr int kNumClass = sizeof(kClassCap) / sizeof(kClassCap[0]);

struct Plan {
    int n_inst = 0;
    InstDev **d_insts = nullptr; // table of the runs' device records
    WorkItem *d_items[kNumClass] = {};
    int n_items[kNumClass] = {};
    int variant[kNumClass] = {};
    // A context's own plan whose cells all take the shared-memory classes
    // keeps room for every cell in every class (class k at d_items_all + k
    // n_cells), so that the device can rebuild it for a new layout
    // (plan_refresh_kernel): refresh[0 .. kNumClass) are then the classes'
    // counts, refresh[kNumClass] = 1 when a cell left those classes.
    bool refreshable = false;
    WorkItem *d_items_all = nullptr;
    uint32_t *d_refresh = nullptr;
    // with several groups of work (size classes, the large-cell path), each
    // size class launches on a stream of its own beside the others
    cudaStream_t cls_side[kNumClass] = {};
    cudaEvent_t cls_fork = nullptr, cls_join[kNumClass] = {};
    cudaStream_t big_hi = nullptr; // then the large-cell path's, at the device's greatest priority
    cudaEvent_t big_join = nullptr;
    WorkItem *d_mid[3] = {};     // cells of the cluster path, by cluster size K = 1, 2, 4, largest first
    int n_mid[3] = {};
    int mid_clusters[3] = {};    // clusters of each launch: the SMs dealt in proportion to the classes' SDs
    cudaStream_t mid_side[3] = {}; // the cluster launches run beside each other and the multi-pass path
    cudaEvent_t mid_fork = nullptr, mid_join[3] = {};
    BigCell *d_bigs = nullptr;
    int n_big = 0;
    BigChunk *d_chunks = nullptr;
    int n_chunks = 0;
    BigBucket *d_buckets = nullptr;
    int n_buckets = 0;
    BigPairs *d_pairs = nullptr;
    int n_pair_blocks = 0;
    BigScratch scratch{};
    int max_big_lb = 0;
    std::vector<Buf> bufs;
    int64_t bytes = 0;
    sdm_tuning tuning{}; // the launch tuning the plan was built with
    std::vector<unsigned char> host_pack; // the tables uploaded in one copy
};

struct SedBuffers;  // second layout and scratch of the sedimentation step (sdm_sediment.cu)
struct CondBuffers; // work list and scratch of the condensation step (sdm_condense.cu)

} // namespace

struct sdm_ctx {
    sdm_config cfg{};
    DevMem mem;
    cudaStream_t stream = nullptr;
    int64_t capacity_sd = 0;
    int64_t n_slots_cap = 0;
    int64_t n_sd = 0;
    int64_t n_slots = 0;
    int64_t step = 0;     // index of the next step
    int64_t dev_base = 0; // value of the device record's step counter
    int32_t largest_cell = 0;
    bool has_attributes = false;
    bool broken = false;
    int64_t layout_version = 0; // changes with every new layout (batches check it)
    // sedimentation: positions set by sdm_set_positions, buffers at first use
    bool has_positions = false;
    int32_t nx = 0;
    double dz = 0.0;
    double *d_zeta = nullptr; // height above the cell's bottom, per slot
    SedBuffers *sed = nullptr;
    CondBuffers *cond = nullptr;
    std::string error;
    // device state
    int64_t *d_xi = nullptr;
    double *d_v = nullptr;
    int32_t *d_id_of_slot = nullptr;
    int32_t *d_cell_off = nullptr;
    InstDev *d_inst = nullptr;
    std::vector<int32_t> h_cell_off;
    // page-locked host staging of sdm_set_attributes' small transfers (the
    // validation block in; offsets and the record out), kept between calls
    unsigned char *h_pin = nullptr;
    size_t h_pin_bytes = 0;
    // page-locked staging of sdm_spectrum (edges and dln in, the status word
    // back), used when the result goes to the host (the call synchronises)
    unsigned char *h_spec = nullptr;
    // copies of host input run on their own stream, in kInChunks pieces, so
    // that each piece is validated while the next one is on its way
    cudaStream_t cstream = nullptr;
    cudaEvent_t in_ev[kInChunks + 1] = {};
    int64_t device_bytes = 0;
    sdm_batch *self_batch = nullptr;
    // pinned host copy of the own batch's launch plan: uploaded from here,
    // written again only after the event shows the last upload done
    void *h_plan = nullptr;
    size_t h_plan_bytes = 0;
    cudaEvent_t plan_ev = nullptr;
};

namespace {
void sed_release(sdm_ctx *ctx);  // frees the sedimentation buffers (sdm_sediment.cu)
void cond_release(sdm_ctx *ctx); // frees the condensation buffers (sdm_condense.cu)
} // namespace

struct sdm_batch {
    std::vector<sdm_ctx *> ctxs;
    cudaStream_t stream = nullptr;
    DevMem mem;
    Plan plan;
    bool use_graph = false;
    int graph_steps = 16;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    int64_t *d_delta = nullptr;       // per-run step deltas for counter syncs
    std::vector<int64_t> h_delta;
    std::vector<int64_t> versions;    // the contexts' layout versions the plan was built for
    sdm_ctx *own = nullptr;           // the context this batch belongs to (sdm_coalescence_step), if any
    std::string error;
    bool broken = false;
};

namespace {

sdm_status fail(std::string *slot, sdm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (slot)
        *slot = buf;
    g_thread_error = buf;
    return st;
}

sdm_status cuda_fail(sdm_ctx *ctx, cudaError_t e, const char *what)
{
    ctx->broken = true;
    return fail(&ctx->error, SDM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

sdm_status cuda_fail(sdm_batch *b, cudaError_t e, const char *what)
{
    b->broken = true;
    for (sdm_ctx *c : b->ctxs)
        c->broken = true;
    return fail(&b->error, SDM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CTX_CUDA(ctx, call)                                                                                            \
    do {                                                                                                               \
        cudaError_t e_ = (call);                                                                                       \
        if (e_ != cudaSuccess)                                                                                         \
            return cuda_fail((ctx), e_, #call);                                                                        \
    } while (0)

template <typename T>
T *plan_alloc(Plan &pl, DevMem &mem, size_t count)
{
    Buf b;
    b.bytes = std::max<size_t>(count * sizeof(T), 16);
    b.p = mem.get(b.bytes);
    if (!b.p)
        return nullptr;
    pl.bufs.push_back(b);
    pl.bytes += (int64_t)b.bytes;
    return static_cast<T *>(b.p);
}

void plan_free(Plan &pl, DevMem &mem)
{
    for (Buf &b : pl.bufs)
        mem.put(b.p, b.bytes);
    for (int k = 0; k < 3; ++k) {
        if (pl.mid_side[k])
            cudaStreamDestroy(pl.mid_side[k]);
        if (pl.mid_join[k])
            cudaEventDestroy(pl.mid_join[k]);
    }
    if (pl.mid_fork)
        cudaEventDestroy(pl.mid_fork);
    for (int k = 0; k < kNumClass; ++k) {
        if (pl.cls_side[k])
            cudaStreamDestroy(pl.cls_side[k]);
        if (pl.cls_join[k])
            cudaEventDestroy(pl.cls_join[k]);
    }
    if (pl.cls_fork)
        cudaEventDestroy(pl.cls_fork);
    if (pl.big_hi)
        cudaStreamDestroy(pl.big_hi);
    if (pl.big_join)
        cudaEventDestroy(pl.big_join);
    pl = Plan{};
}

int big_lb(int n)
{
    int lg = 0;
    while ((1 << lg) < n)
        ++lg;
    return std::min(std::max(lg - 10, 1), kBigMaxLB);
}

size_t big_hist_smem(int lb) { return (size_t)sizeof(uint32_t) << lb; }

// Kernel variants of the shared-memory path.  Warp-per-cell kernels for cells
// of up to 256 SDs (capacity, warps per block; 2 pipeline stages); block-per-
// cell kernels for every class (capacity, threads, stages).  The launch
// tuning (sdm_set_tuning) picks one variant per size class when a plan is
// built.
#define SDM_WARP_VARIANTS(X)                                                                                           \
    X(64, 1) X(64, 2) X(64, 4) X(128, 1) X(128, 2) X(128, 4) X(256, 1) X(256, 2) X(256, 4) X(512, 1) X(512, 2) X(512, 4)
#define SDM_BLOCK_VARIANTS(X)                                                                                          \
    X(64, 32, 4) X(128, 64, 4) X(256, 128, 4) X(512, 256, 4) X(1024, 512, 3) X(2048, 1024, 2) X(4096, 1024, 2)

typedef void (*launch_fn)(int grid, int n, const WorkItem *, InstDev *const *, int64_t, cudaStream_t);

template <int CAP, int WARPS>
void launch_warp(int grid, int n, const WorkItem *items, InstDev *const *insts, int64_t off, cudaStream_t st)
{
    warp_cell_step_kernel<CAP, WARPS, 2><<<grid, 32 * WARPS, WarpSmem<CAP, 2>::per_warp * WARPS, st>>>(items, n, insts,
                                                                                                     off);
}

// The fused form (every cell stays in shared memory for nf steps) always runs
// 2 warps per block, with one pipeline stage per warp: a warp loads a cell
// once per nf steps, so a second stage would only cost shared memory.
template <int CAP>
void launch_warp_fused(int grid, int n, const WorkItem *items, InstDev *const *insts, int64_t off, int32_t nf,
                       cudaStream_t st)
{
    warp_cell_step_kernel<CAP, 2, 1, true><<<grid, 64, WarpSmem<CAP, 1>::per_warp * 2, st>>>(items, n, insts, off, nf);
}

template <int CAP, int NT, int ST>
void launch_block(int grid, int n, const WorkItem *items, InstDev *const *insts, int64_t off, cudaStream_t st)
{
    cell_step_kernel<CAP, NT, ST><<<grid, NT, CellSmem<CAP, ST>::bytes, st>>>(items, n, insts, off);
}

typedef void (*fused_fn)(int grid, int n, const WorkItem *, InstDev *const *, int64_t, int32_t, cudaStream_t);

struct Variant {
    int cap;
    int warps; // warps per block of the warp kernel; 0: block kernel
    launch_fn launch;
};

// the fused warp kernels by capacity 64 .. 512
struct FusedVariant {
    int cap;
    fused_fn launch;
};
const FusedVariant g_fused[] = {{64, launch_warp_fused<64>},
                                {128, launch_warp_fused<128>},
                                {256, launch_warp_fused<256>},
                                {512, launch_warp_fused<512>}};

const Variant g_variants[] = {
#define X(CAP, WARPS) {CAP, WARPS, launch_warp<CAP, WARPS>},
    SDM_WARP_VARIANTS(X)
#undef X
#define X(CAP, NT, ST) {CAP, 0, launch_block<CAP, NT, ST>},
        SDM_BLOCK_VARIANTS(X)
#undef X
};
constexpr int kNumVariants = sizeof(g_variants) / sizeof(g_variants[0]);
constexpr int kNumFused = sizeof(g_fused) / sizeof(g_fused[0]);
constexpr int kMaxDevices = 64;

// Per-device launch set-up: the kernels' shared-memory limits are attributes
// of each device's context, and the persistent grids are sized from that
// device's SM count (resident blocks x SMs).
struct DevGrids {
    bool done = false;
    cudaError_t status = cudaSuccess;
    int variant[kNumVariants] = {};
    int fused[kNumFused] = {};
    int mid[3] = {}; // clusters of the mid-size-cell kernel resident at once, K = 1, 2, 4
    int spec = 1;    // blocks of the total-spectrum kernel
};
std::mutex g_dev_mutex;
DevGrids g_dev[kMaxDevices];

// The current device's table (configured by configure_kernels).
const DevGrids &dev_grids()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        dev = 0;
    return g_dev[dev];
}

std::mutex g_tuning_mutex;
sdm_tuning g_tuning = {4096, 512, 2, SDM_FUSE_STEPS_DEFAULT, SDM_MID_MAX_SD_DEFAULT};

bool same_tuning(const sdm_tuning &a, const sdm_tuning &b)
{
    return a.smem_max_sd == b.smem_max_sd && a.warp_cell_max == b.warp_cell_max &&
           a.warps_per_block == b.warps_per_block && a.fuse_steps == b.fuse_steps && a.mid_max_sd == b.mid_max_sd;
}

sdm_tuning current_tuning()
{
    std::lock_guard<std::mutex> lock(g_tuning_mutex);
    return g_tuning;
}

int variant_for(int cap, const sdm_tuning &t)
{
    for (int v = 0; v < kNumVariants; ++v) {
        const Variant &x = g_variants[v];
        if (x.cap != cap)
            continue;
        if (cap <= t.warp_cell_max ? x.warps == t.warps_per_block : x.warps == 0)
            return v;
    }
    return -1;
}

// The mid-size-cell kernel with K CTAs per cluster: its shared-memory limit,
// and how many clusters fit on the device at once (its persistent grid).
template <int K>
cudaError_t mid_configure(int &clusters)
{
    cudaError_t r = cudaFuncSetAttribute(mid_cell_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)MidSmem<K>::bytes);
    if (r != cudaSuccess)
        return r;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(K, 1, 1);
    cfg.blockDim = dim3(kMidNT, 1, 1);
    cfg.dynamicSmemBytes = MidSmem<K>::bytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    r = cudaOccupancyMaxActiveClusters(&n, mid_cell_kernel<K>, &cfg);
    clusters = n > 0 ? n : 1;
    return r;
}

template <int K>
cudaError_t launch_mid(int clusters, int n, const WorkItem *items, InstDev *const *insts, int64_t off, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(K * clusters, 1, 1);
    cfg.blockDim = dim3(kMidNT, 1, 1);
    cfg.dynamicSmemBytes = MidSmem<K>::bytes;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, mid_cell_kernel<K>, items, (int32_t)n, insts, off);
}

// Configures the current device once (the first context, batch or spectrum
// call on each device does it, with that device current).
cudaError_t configure_kernels()
{
    int dev = 0;
    cudaError_t r = cudaGetDevice(&dev);
    if (r != cudaSuccess)
        return r;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    DevGrids &G = g_dev[dev];
    if (G.done)
        return G.status;
    G.status = [&] {
        cudaError_t e = cudaSuccess;
        int sms = 0;
        if ((r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return r;
        int v = 0;
#define X(CAP, WARPS)                                                                                                  \
    {                                                                                                                  \
        const int bytes = (int)(WarpSmem<CAP, 2>::per_warp * WARPS);                                                   \
        if ((r = cudaFuncSetAttribute(warp_cell_step_kernel<CAP, WARPS, 2>,                                            \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)             \
            e = r;                                                                                                     \
        int per_sm = 0;                                                                                                \
        if ((r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, warp_cell_step_kernel<CAP, WARPS, 2>,          \
                                                               32 * WARPS, bytes)) != cudaSuccess)                     \
            e = r;                                                                                                     \
        G.variant[v++] = std::max(1, per_sm) * sms;                                                                   \
    }
        SDM_WARP_VARIANTS(X)
#undef X
#define X(CAP, NT, ST)                                                                                                 \
    {                                                                                                                  \
        const int bytes = (int)CellSmem<CAP, ST>::bytes;                                                               \
        if ((r = cudaFuncSetAttribute(cell_step_kernel<CAP, NT, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                      bytes)) != cudaSuccess)                                                          \
            e = r;                                                                                                     \
        int per_sm = 0;                                                                                                \
        if ((r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cell_step_kernel<CAP, NT, ST>, NT, bytes)) != \
            cudaSuccess)                                                                                               \
            e = r;                                                                                                     \
        G.variant[v++] = std::max(1, per_sm) * sms;                                                                   \
    }
        SDM_BLOCK_VARIANTS(X)
#undef X
        v = 0;
#define X(CAP)                                                                                                         \
    {                                                                                                                  \
        const int bytes = (int)(WarpSmem<CAP, 1>::per_warp * 2);                                                       \
        if ((r = cudaFuncSetAttribute(warp_cell_step_kernel<CAP, 2, 1, true>,                                          \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)             \
            e = r;                                                                                                     \
        int per_sm = 0;                                                                                                \
        if ((r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, warp_cell_step_kernel<CAP, 2, 1, true>, 64,    \
                                                               bytes)) != cudaSuccess)                                 \
            e = r;                                                                                                     \
        G.fused[v++] = std::max(1, per_sm) * sms;                                                                      \
    }
        X(64) X(128) X(256) X(512)
#undef X
        int spec_per_sm = 0;
        if ((r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&spec_per_sm, spectrum_total_kernel, kSpecTotNT, 0)) !=
            cudaSuccess)
            e = r;
        G.spec = std::max(1, spec_per_sm) * sms;
        const int hb = (int)big_hist_smem(kBigMaxLB);
        if ((r = cudaFuncSetAttribute(big_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, hb)) != cudaSuccess) e = r;
        if ((r = cudaFuncSetAttribute(big_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, hb)) != cudaSuccess) e = r;
        if ((r = cudaFuncSetAttribute(big_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, hb)) != cudaSuccess) e = r;
        if ((r = mid_configure<1>(G.mid[0])) != cudaSuccess) e = r;
        if ((r = mid_configure<2>(G.mid[1])) != cudaSuccess) e = r;
        if ((r = mid_configure<4>(G.mid[2])) != cudaSuccess) e = r;
        return e;
    }();
    G.done = true;
    return G.status;
}

void launch_variant(int v, int n, const WorkItem *items, InstDev *const *insts, int64_t off, cudaStream_t st)
{
    const Variant &x = g_variants[v];
    const int per_block = x.warps > 0 ? x.warps : 1;
    const int grid = std::min((n + per_block - 1) / per_block, dev_grids().variant[v]);
    x.launch(grid, n, items, insts, off, st);
}

// Size class of a cell of n >= 2 stored SDs under the tuning (the smallest
// class capacity 64 2^c >= n); -1: the multi-pass path.
int class_of(int n, const sdm_tuning &t)
{
    const int c = n <= 64 ? 0 : 32 - __builtin_clz((unsigned)(n - 1)) - 6;
    if (c >= kNumClass || kClassCap[c] > t.smem_max_sd)
        return -1;
    return c;
}

constexpr int kRefreshNT = 256;

// The work items of a run whose cells all take the shared-memory classes,
// from its cell offsets, as build_plan makes them (class_of): class k's at
// items + k cap, their number added to counts[k]; counts[kNumClass] = 1 when
// a cell is above smem_max_sd.  Block-level counts first, then one global
// atomic per class and block (the order of a class's items is free: cells
// are independent).
__global__ void __launch_bounds__(kRefreshNT) plan_refresh_kernel(const int32_t *__restrict__ cell_off,
                                                                  int32_t n_cells, int32_t cell_base,
                                                                  int32_t smem_max_sd, WorkItem *__restrict__ items,
                                                                  int32_t cap, uint32_t *__restrict__ counts)
{
    __shared__ uint32_t s_cnt[kNumClass], s_base[kNumClass];
    if (threadIdx.x < kNumClass)
        s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    const int c = blockIdx.x * kRefreshNT + threadIdx.x;
    int k = -1, o = 0, n = 0;
    uint32_t slot = 0;
    if (c < n_cells) {
        o = cell_off[c];
        n = cell_off[c + 1] - o;
        if (n >= 2) {
            k = n <= 64 ? 0 : 32 - __clz(n - 1) - 6;
            if (k >= kNumClass || (64 << k) > smem_max_sd) {
                counts[kNumClass] = 1u;
                k = -1;
            } else {
                slot = atomicAdd(&s_cnt[k], 1u);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < kNumClass)
        s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(&counts[threadIdx.x], s_cnt[threadIdx.x]) : 0u;
    __syncthreads();
    if (k >= 0)
        items[(int64_t)k * cap + s_base[k] + slot] = WorkItem{0, cell_base + c, o, n};
}

// Starts the device rebuild of a refreshable plan from the run's offsets.
cudaError_t plan_refresh(Plan &pl, const int32_t *d_cell_off, int32_t n_cells, int32_t cell_base, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(pl.d_refresh, 0, sizeof(uint32_t) * (kNumClass + 1), st);
    if (e != cudaSuccess || n_cells == 0)
        return e;
    plan_refresh_kernel<<<(n_cells + kRefreshNT - 1) / kRefreshNT, kRefreshNT, 0, st>>>(
        d_cell_off, n_cells, cell_base, pl.tuning.smem_max_sd, pl.d_items_all, n_cells, pl.d_refresh);
    return cudaGetLastError();
}

// Work lists of every run in the batch, split by cell size.
sdm_status build_plan(sdm_batch *b)
{
    Plan &pl = b->plan;
    DevMem &mem = b->mem;
    const int n_inst = (int)b->ctxs.size();
    // the tables are gathered in host vectors kept by the thread, so that a
    // plan rebuilt after every sedimentation step reuses their memory
    struct Scratch {
        std::vector<WorkItem> items[kNumClass];
        std::vector<WorkItem> mid[3];
        std::vector<BigCell> bigs;
        std::vector<BigChunk> chunks;
        std::vector<BigBucket> buckets;
        std::vector<BigPairs> pairs;
        std::vector<InstDev *> insts;
        std::vector<int8_t> cls; // per cell of a run: its class, -1 above them, -2 fewer than 2 SDs
    };
    static thread_local Scratch scr;
    std::vector<WorkItem>(&items)[kNumClass] = scr.items;
    std::vector<WorkItem>(&mid)[3] = scr.mid;
    std::vector<BigCell> &bigs = scr.bigs;
    std::vector<BigChunk> &chunks = scr.chunks;
    std::vector<BigBucket> &buckets = scr.buckets;
    std::vector<BigPairs> &pairs = scr.pairs;
    std::vector<InstDev *> &insts = scr.insts;
    for (auto &v : items)
        v.clear();
    for (auto &v : mid)
        v.clear();
    bigs.clear();
    chunks.clear();
    buckets.clear();
    pairs.clear();
    insts.assign(n_inst, nullptr);
    int64_t hist_total = 0, sd_total = 0, bkt_total = 0;
    const sdm_tuning tun = current_tuning();
    pl.tuning = tun;
    for (int k = 0; k < kNumClass; ++k)
        pl.variant[k] = variant_for(kClassCap[k], tun);
    for (int i = 0; i < n_inst; ++i) {
        sdm_ctx *c = b->ctxs[i];
        insts[i] = c->d_inst;
        const int32_t *off = c->h_cell_off.data();
        const int32_t nc = c->cfg.n_cells, cb = c->cfg.cell_base;
        // the shared-memory classes in two tight passes (a class per cell and
        // the classes' sizes, then the items into their places); the other
        // cells after
        std::vector<int8_t> &cls = scr.cls;
        cls.resize((size_t)nc);
        size_t cnt[kNumClass] = {};
        bool above = false;
        for (int32_t cell = 0; cell < nc; ++cell) {
            const int n = off[cell + 1] - off[cell];
            const int8_t k = n < 2 ? (int8_t)-2 : (int8_t)class_of(n, tun);
            cls[cell] = k;
            if (k >= 0)
                ++cnt[k];
            above |= k == -1;
        }
        WorkItem *dst[kNumClass];
        for (int k = 0; k < kNumClass; ++k) {
            const size_t at = items[k].size();
            items[k].resize(at + cnt[k]);
            dst[k] = items[k].data() + at;
        }
        for (int32_t cell = 0; cell < nc; ++cell) {
            const int k = cls[cell];
            if (k >= 0)
                *dst[k]++ = WorkItem{i, cb + cell, off[cell], off[cell + 1] - off[cell]};
        }
        if (!above)
            continue;
        for (int cell = 0; cell < nc; ++cell) {
            if (cls[cell] != -1)
                continue;
            const int n = off[cell + 1] - off[cell];
            if (n <= tun.mid_max_sd) { // the cluster path, K = 1, 2 or 4 CTAs (sorted below)
                const int km = n <= kMidSdPerCta ? 0 : (n <= 2 * kMidSdPerCta ? 1 : 2);
                mid[km].push_back(WorkItem{i, c->cfg.cell_base + cell, c->h_cell_off[cell], n});
                continue;
            }
            BigCell bc{};
            bc.inst = i;
            bc.cell = cell;
            bc.rcell = c->cfg.cell_base + cell;
            bc.n = n;
            bc.lb = big_lb(n);
            bc.n_chunks = (n + kBigChunk - 1) / kBigChunk;
            bc.hist_base = hist_total;
            bc.sd_base = sd_total;
            bc.bkt_base = bkt_total;
            hist_total += (int64_t)bc.n_chunks << bc.lb;
            sd_total += n;
            bkt_total += (1 << bc.lb) + 1;
            const int big = (int)bigs.size();
            for (int k = 0; k < bc.n_chunks; ++k)
                chunks.push_back(BigChunk{big, k});
            for (int k = 0; k < (1 << bc.lb); ++k)
                buckets.push_back(BigBucket{big, k});
            const int n_q = (n / 2 + 1) / 2; // pair-of-pairs upper bound
            for (int q0 = 0; q0 < n_q; q0 += kPairNT)
                pairs.push_back(BigPairs{big, q0});
            pl.max_big_lb = std::max(pl.max_big_lb, bc.lb);
            bigs.push_back(bc);
        }
    }
    for (int k = 0; k < 3; ++k) // largest cells first (the kernel deals them in a snake order)
        std::stable_sort(mid[k].begin(), mid[k].end(), [](const WorkItem &a, const WorkItem &c) { return a.n > c.n; });
    // every table (the runs, the work list of each class, the big-cell
    // descriptors) in one host buffer, one device buffer and one copy
    pl.n_inst = n_inst;
    auto a16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
    size_t off_items[kNumClass], sz = a16(sizeof(InstDev *) * n_inst);
    for (int k = 0; k < kNumClass; ++k) {
        off_items[k] = sz;
        sz += a16(sizeof(WorkItem) * items[k].size());
    }
    size_t off_mid[3];
    for (int k = 0; k < 3; ++k) {
        off_mid[k] = sz;
        sz += a16(sizeof(WorkItem) * mid[k].size());
    }
    const size_t off_bigs = sz;
    sz += a16(sizeof(BigCell) * bigs.size());
    const size_t off_chunks = sz;
    sz += a16(sizeof(BigChunk) * chunks.size());
    const size_t off_buckets = sz;
    sz += a16(sizeof(BigBucket) * buckets.size());
    const size_t off_pairs = sz;
    sz += a16(sizeof(BigPairs) * pairs.size());
    // the own batch of a context uploads from the context's pinned copy (its
    // last upload done first); other batches from a host vector of the plan
    unsigned char *h = nullptr;
    sdm_ctx *own = b->own;
    if (own) {
        if (own->plan_ev)
            cudaEventSynchronize(own->plan_ev);
        if (own->h_plan_bytes < sz) {
            if (own->h_plan)
                cudaFreeHost(own->h_plan);
            own->h_plan = nullptr;
            own->h_plan_bytes = 0;
            const size_t want = sz + sz / 4 + 4096;
            if (cudaMallocHost(&own->h_plan, want) == cudaSuccess)
                own->h_plan_bytes = want;
            else
                cudaGetLastError();
        }
        if (own->h_plan && !own->plan_ev &&
            cudaEventCreateWithFlags(&own->plan_ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            own->plan_ev = nullptr;
        }
        if (own->h_plan && own->plan_ev)
            h = static_cast<unsigned char *>(own->h_plan);
    }
    if (!h) {
        pl.host_pack.assign(sz, 0);
        h = pl.host_pack.data();
    }
    std::memcpy(h, insts.data(), sizeof(InstDev *) * n_inst);
    for (int k = 0; k < kNumClass; ++k)
        if (!items[k].empty())
            std::memcpy(h + off_items[k], items[k].data(), sizeof(WorkItem) * items[k].size());
    for (int k = 0; k < 3; ++k)
        if (!mid[k].empty())
            std::memcpy(h + off_mid[k], mid[k].data(), sizeof(WorkItem) * mid[k].size());
    if (!bigs.empty()) {
        std::memcpy(h + off_bigs, bigs.data(), sizeof(BigCell) * bigs.size());
        std::memcpy(h + off_chunks, chunks.data(), sizeof(BigChunk) * chunks.size());
        std::memcpy(h + off_buckets, buckets.data(), sizeof(BigBucket) * buckets.size());
        std::memcpy(h + off_pairs, pairs.data(), sizeof(BigPairs) * pairs.size());
    }
    unsigned char *d = plan_alloc<unsigned char>(pl, mem, sz);
    if (!d)
        return fail(&b->error, SDM_ENOMEM, "batch plan: device allocation failed");
    pl.d_insts = reinterpret_cast<InstDev **>(d);
    for (int k = 0; k < kNumClass; ++k) {
        pl.n_items[k] = (int)items[k].size();
        pl.d_items[k] = pl.n_items[k] ? reinterpret_cast<WorkItem *>(d + off_items[k]) : nullptr;
    }
    // a context's own plan of shared-memory classes only: items with room
    // for every cell in every class, built on the device like later refreshes
    if (own && n_inst == 1 && bigs.empty() && mid[0].empty() && mid[1].empty() && mid[2].empty()) {
        const int32_t nc = own->cfg.n_cells;
        pl.d_items_all = plan_alloc<WorkItem>(pl, mem, (size_t)kNumClass * std::max(nc, 1));
        pl.d_refresh = plan_alloc<uint32_t>(pl, mem, kNumClass + 1);
        if (!pl.d_items_all || !pl.d_refresh)
            return fail(&b->error, SDM_ENOMEM, "batch plan: device allocation failed");
        pl.refreshable = true;
        for (int k = 0; k < kNumClass; ++k)
            pl.d_items[k] = pl.d_items_all + (size_t)k * nc;
        const cudaError_t e = plan_refresh(pl, own->d_cell_off, nc, own->cfg.cell_base, b->stream);
        if (e != cudaSuccess)
            return cuda_fail(b, e, "batch plan: work items");
    }
    for (int k = 0; k < 3; ++k) {
        pl.n_mid[k] = (int)mid[k].size();
        pl.d_mid[k] = pl.n_mid[k] ? reinterpret_cast<WorkItem *>(d + off_mid[k]) : nullptr;
    }
    {
        // the device's SMs (one cluster-path CTA each) dealt to the classes in
        // proportion to their SDs (the multi-pass path's cells, which run beside
        // them, count too), at least one cluster to each class with cells, at
        // most one per cell and no more than fit at once
        const DevGrids &G = dev_grids();
        int64_t work[3] = {}, total = sd_total;
        for (int k = 0; k < 3; ++k) {
            for (const WorkItem &w : mid[k])
                work[k] += w.n;
            total += work[k];
        }
        const int ks[3] = {1, 2, 4};
        const int sms = G.mid[0];
        for (int k = 0; k < 3; ++k) {
            if (!pl.n_mid[k])
                continue;
            const int share = (int)((double)sms * (double)work[k] / (double)total) / ks[k];
            pl.mid_clusters[k] = std::max(1, std::min({share, pl.n_mid[k], G.mid[k]}));
        }
        int classes = bigs.empty() ? 0 : 1;
        for (int k = 0; k < 3; ++k)
            classes += pl.n_mid[k] ? 1 : 0;
        if (classes > 1) {
            cudaError_t e = cudaEventCreateWithFlags(&pl.mid_fork, cudaEventDisableTiming);
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
                e = cudaStreamCreateWithFlags(&pl.mid_side[k], cudaStreamNonBlocking);
                if (e == cudaSuccess)
                    e = cudaEventCreateWithFlags(&pl.mid_join[k], cudaEventDisableTiming);
            }
            if (e != cudaSuccess)
                return cuda_fail(b, e, "batch plan: side streams");
        }
        // the size classes side by side when there is more than one group of
        // work: those whose cells do not fill the device's resident blocks on
        // their own (a class that fills them gains nothing beside another),
        // and not when the multi-pass path holds more than 2^22 SDs (it then
        // fills the device by itself, and the classes beside it only slowed
        // it: 1.64e10 against 1.67e10 pair-updates/s on the 1024-box ensemble,
        // while mixes of a few dozen runs stepped a third faster)
        bool small[kNumClass] = {};
        int groups = classes > 0 ? 1 : 0;
        for (int k = 0; k < kNumClass; ++k) {
            if (!pl.n_items[k])
                continue;
            ++groups;
            const Variant &x = g_variants[pl.variant[k]];
            small[k] = (int64_t)pl.n_items[k] < (int64_t)G.variant[pl.variant[k]] * (x.warps > 0 ? x.warps : 1);
        }
        if (groups > 1 && sd_total <= ((int64_t)1 << 22)) {
            cudaError_t e = cudaEventCreateWithFlags(&pl.cls_fork, cudaEventDisableTiming);
            for (int k = 0; k < kNumClass && e == cudaSuccess; ++k) {
                if (!small[k])
                    continue;
                e = cudaStreamCreateWithFlags(&pl.cls_side[k], cudaStreamNonBlocking);
                if (e == cudaSuccess)
                    e = cudaEventCreateWithFlags(&pl.cls_join[k], cudaEventDisableTiming);
            }
            // the large-cell path (the critical one when present) ahead of the
            // forked classes in the block scheduler
            if (e == cudaSuccess && classes > 0) {
                int least = 0, greatest = 0;
                e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
                if (e == cudaSuccess)
                    e = cudaStreamCreateWithPriority(&pl.big_hi, cudaStreamNonBlocking, greatest);
                if (e == cudaSuccess)
                    e = cudaEventCreateWithFlags(&pl.big_join, cudaEventDisableTiming);
            }
            if (e != cudaSuccess)
                return cuda_fail(b, e, "batch plan: size-class streams");
        }
    }
    if (!bigs.empty()) {
        pl.n_big = (int)bigs.size();
        pl.n_chunks = (int)chunks.size();
        pl.n_buckets = (int)buckets.size();
        pl.n_pair_blocks = (int)pairs.size();
        pl.d_bigs = reinterpret_cast<BigCell *>(d + off_bigs);
        pl.d_chunks = reinterpret_cast<BigChunk *>(d + off_chunks);
        pl.d_buckets = reinterpret_cast<BigBucket *>(d + off_buckets);
        pl.d_pairs = reinterpret_cast<BigPairs *>(d + off_pairs);
        pl.scratch.hist = plan_alloc<uint32_t>(pl, mem, hist_total);
        pl.scratch.bstart = plan_alloc<uint32_t>(pl, mem, bkt_total);
        pl.scratch.rank = plan_alloc<uint32_t>(pl, mem, sd_total);
        pl.scratch.perm = plan_alloc<uint32_t>(pl, mem, sd_total);
        pl.scratch.scale = plan_alloc<double>(pl, mem, bigs.size());
        pl.scratch.scale_f = plan_alloc<float>(pl, mem, bigs.size());
        pl.scratch.live = plan_alloc<uint32_t>(pl, mem, chunks.size() * kLiveWords);
        if (!pl.scratch.hist || !pl.scratch.bstart || !pl.scratch.rank || !pl.scratch.perm ||
            !pl.scratch.scale || !pl.scratch.scale_f || !pl.scratch.live)
            return fail(&b->error, SDM_ENOMEM, "batch plan: big-cell scratch allocation failed");
    }
    // the host copy lives as long as the plan (or, pinned, until the event
    // below has passed): no wait for the upload
    cudaError_t e = cudaMemcpyAsync(d, h, sz, cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess)
        return cuda_fail(b, e, "batch plan upload");
    if (own && h == own->h_plan && (e = cudaEventRecord(own->plan_ev, b->stream)) != cudaSuccess)
        return cuda_fail(b, e, "batch plan upload event");
    return SDM_OK;
}

// n steps (offsets off .. off + n - 1 from each run's device counter) of
// every cell above the shared-memory threshold: the cluster path and the
// multi-pass path.  The cluster sizes run side by side and beside the
// multi-pass path (one fork and one join by events for all n steps; a graph
// captures the same), each cluster size on its share of the SMs, the
// multi-pass kernels on the rest; a cluster size's steps follow each other
// on its stream, and the multi-pass path's on st.
void enqueue_big_steps(const Plan &pl, int64_t off, int32_t n, cudaStream_t st)
{
    const bool fork = pl.mid_fork != nullptr;
    if (fork) {
        cudaEventRecord(pl.mid_fork, st);
        for (int k = 0; k < 3; ++k)
            if (pl.n_mid[k])
                cudaStreamWaitEvent(pl.mid_side[k], pl.mid_fork, 0);
    }
    auto side = [&](int k) { return fork ? pl.mid_side[k] : st; };
    for (int32_t i = 0; i < n; ++i) {
        if (pl.n_mid[2])
            launch_mid<4>(pl.mid_clusters[2], pl.n_mid[2], pl.d_mid[2], pl.d_insts, off + i, side(2));
        if (pl.n_mid[1])
            launch_mid<2>(pl.mid_clusters[1], pl.n_mid[1], pl.d_mid[1], pl.d_insts, off + i, side(1));
        if (pl.n_mid[0])
            launch_mid<1>(pl.mid_clusters[0], pl.n_mid[0], pl.d_mid[0], pl.d_insts, off + i, side(0));
    }
    for (int32_t i = 0; pl.n_big && i < n; ++i) {
        const int64_t o = off + i;
        const size_t hs = big_hist_smem(pl.max_big_lb);
        big_hist_kernel<<<pl.n_chunks, kBigNT, hs, st>>>(pl.d_chunks, pl.d_bigs, pl.d_insts, pl.scratch, o);
        const int tiles = std::max(1, (1 << pl.max_big_lb) / kBigColNT);
        big_colscan_kernel<<<pl.n_big * tiles, kBigColNT, 0, st>>>(pl.d_bigs, tiles, pl.scratch);
        big_scan_kernel<<<pl.n_big, kBigNT, big_hist_smem(kBigMaxLB), st>>>(pl.d_bigs, pl.d_insts, pl.scratch);
        big_scatter_kernel<<<pl.n_chunks, kBigNT, hs, st>>>(pl.d_chunks, pl.d_bigs, pl.d_insts, pl.scratch, o);
        big_bucket_sort_kernel<<<pl.n_buckets, kBucketNT, 0, st>>>(pl.d_buckets, pl.d_bigs, pl.d_insts, pl.scratch,
                                                                   o);
        big_pairs_kernel<<<pl.n_pair_blocks, kPairNT, 0, st>>>(pl.d_pairs, pl.d_bigs, pl.d_insts, pl.scratch, o);
    }
    if (fork)
        for (int k = 0; k < 3; ++k)
            if (pl.n_mid[k]) {
                cudaEventRecord(pl.mid_join[k], pl.mid_side[k]);
                cudaStreamWaitEvent(st, pl.mid_join[k], 0);
            }
}

// The size classes' launches on their own streams (forked from st, joined
// back by join()), when the plan has them; else, and for a class that a
// refresh of the plan on the device filled after it was built, on st.
struct ClassFork {
    const Plan &pl;
    cudaStream_t st;
    bool on;
    ClassFork(const Plan &p, cudaStream_t s) : pl(p), st(s), on(p.cls_fork != nullptr)
    {
        if (!on)
            return;
        cudaEventRecord(pl.cls_fork, st);
        for (int k = 0; k < kNumClass; ++k)
            if (side(k))
                cudaStreamWaitEvent(pl.cls_side[k], pl.cls_fork, 0);
    }
    bool side(int k) const { return on && pl.n_items[k] && pl.cls_side[k]; }
    cudaStream_t of(int k) const { return side(k) ? pl.cls_side[k] : st; }
    // the stream of the large-cell path (forked at the same point)
    cudaStream_t big() const
    {
        if (!on || !pl.big_hi)
            return st;
        cudaStreamWaitEvent(pl.big_hi, pl.cls_fork, 0);
        return pl.big_hi;
    }
    void join() const
    {
        for (int k = 0; k < kNumClass; ++k)
            if (side(k)) {
                cudaEventRecord(pl.cls_join[k], pl.cls_side[k]);
                cudaStreamWaitEvent(st, pl.cls_join[k], 0);
            }
        if (on && pl.big_hi) {
            cudaEventRecord(pl.big_join, pl.big_hi);
            cudaStreamWaitEvent(st, pl.big_join, 0);
        }
    }
};

// Enqueues n steps (offsets off .. off + n - 1) of every cell.  Cells are
// independent, so each one may take its n steps apart from the others: with
// fusion on (tuning fuse_steps f >= 2) the warp-per-cell classes take up to f
// steps per launch, the other cells one launch per step.
void enqueue_steps(const Plan &pl, int64_t off, int32_t n, cudaStream_t st)
{
    // one fork and one join for all n steps: every class's launches follow
    // each other on its stream, the large-cell path's on its own, and no
    // class waits for another between steps (their cells are independent)
    const ClassFork cf(pl, st);
    const cudaStream_t bs = cf.big();
    const int32_t f = pl.tuning.fuse_steps;
    const bool fuse = f >= 2 && n >= 2;
    for (int k = 0; k < kNumClass; ++k) {
        if (!pl.n_items[k])
            continue;
        const Variant &x = g_variants[pl.variant[k]];
        if (fuse && x.warps > 0) {
            const FusedVariant &fv = g_fused[k];
            const int grid = std::min((pl.n_items[k] + 1) / 2, dev_grids().fused[k]);
            for (int32_t i = 0; i < n; i += f)
                fv.launch(grid, pl.n_items[k], pl.d_items[k], pl.d_insts, off + i, std::min(f, n - i), cf.of(k));
        } else {
            for (int32_t i = 0; i < n; ++i)
                launch_variant(pl.variant[k], pl.n_items[k], pl.d_items[k], pl.d_insts, off + i, cf.of(k));
        }
    }
    enqueue_big_steps(pl, off, n, bs);
    cf.join();
}

// A captured graph: n steps from the device counters, then the counters advance by n.
void enqueue_graph_body(const Plan &pl, int32_t n, cudaStream_t st)
{
    enqueue_steps(pl, 0, n, st);
    advance_steps_kernel<<<(pl.n_inst + 255) / 256, 256, 0, st>>>(pl.d_insts, pl.n_inst, n, nullptr);
}

// Brings every run's device counter up to its host step.
sdm_status sync_counters(sdm_batch *b)
{
    bool any = false;
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        b->h_delta[i] = b->ctxs[i]->step - b->ctxs[i]->dev_base;
        any |= b->h_delta[i] != 0;
    }
    if (!any)
        return SDM_OK;
    cudaError_t e = cudaMemcpyAsync(b->d_delta, b->h_delta.data(), sizeof(int64_t) * b->ctxs.size(),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess)
        return cuda_fail(b, e, "step counter sync");
    advance_steps_kernel<<<(b->plan.n_inst + 255) / 256, 256, 0, b->stream>>>(b->plan.d_insts, b->plan.n_inst, 0,
                                                                              b->d_delta);
    for (sdm_ctx *c : b->ctxs)
        c->dev_base = c->step;
    return SDM_OK;
}

sdm_status batch_init(sdm_batch *b, sdm_ctx *const *ctxs, int32_t n_ctx, cudaStream_t stream, int use_graph,
                      int graph_steps)
{
    for (int i = 0; i < n_ctx; ++i) {
        if (!ctxs[i])
            return fail(&b->error, SDM_EINVAL, "context %d is NULL", i);
        if (ctxs[i]->broken)
            return fail(&b->error, SDM_ESTATE, "context %d is unusable after a CUDA error", i);
        if (!ctxs[i]->has_attributes)
            return fail(&b->error, SDM_ESTATE, "context %d has no attributes", i);
        b->ctxs.push_back(ctxs[i]);
        b->versions.push_back(ctxs[i]->layout_version);
    }
    b->stream = stream;
    b->mem.use_hooks_of(ctxs[0]->mem, stream);
    b->use_graph = use_graph != 0;
    b->graph_steps = graph_steps > 0 ? graph_steps : 16;
    cudaError_t e = configure_kernels();
    if (e != cudaSuccess)
        return cuda_fail(b, e, "kernel configuration");
    sdm_status st = build_plan(b);
    if (st != SDM_OK)
        return st;
    b->h_delta.assign(b->ctxs.size(), 0);
    b->d_delta = plan_alloc<int64_t>(b->plan, b->mem, b->ctxs.size());
    if (!b->d_delta)
        return fail(&b->error, SDM_ENOMEM, "batch: device allocation failed");
    return SDM_OK;
}

void batch_release(sdm_batch *b)
{
    if (b->graph_exec)
        cudaGraphExecDestroy(b->graph_exec);
    if (b->capture_stream)
        cudaStreamDestroy(b->capture_stream);
    b->graph_exec = nullptr;
    b->capture_stream = nullptr;
    plan_free(b->plan, b->mem);
    b->mem.release_kept();
}

sdm_status batch_step(sdm_batch *b, int32_t n_steps)
{
    if (b->broken)
        return fail(&b->error, SDM_ESTATE, "batch unusable after a CUDA error");
    if (n_steps < 0)
        return fail(&b->error, SDM_EINVAL, "n_steps < 0");
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        if (b->ctxs[i]->broken)
            return fail(&b->error, SDM_ESTATE, "a context of the batch is unusable");
        if (b->ctxs[i]->layout_version != b->versions[i])
            return fail(&b->error, SDM_ESTATE,
                        "context %zu has a new layout (set_attributes or a sedimentation step): create the batch again",
                        i);
    }
    if (n_steps == 0)
        return SDM_OK;
    int32_t left = n_steps;
    // direct launches need one common offset (host step - device counter)
    const int64_t pend = b->ctxs[0]->step - b->ctxs[0]->dev_base;
    bool uniform = true;
    for (sdm_ctx *c : b->ctxs)
        uniform &= (c->step - c->dev_base) == pend;
    const bool graph = b->use_graph && n_steps >= b->graph_steps;
    if (graph || !uniform) {
        sdm_status st = sync_counters(b);
        if (st != SDM_OK)
            return st;
    }
    if (graph) {
        if (!b->graph_exec) {
            cudaError_t e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess)
                return cuda_fail(b, e, "graph capture stream");
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess)
                return cuda_fail(b, e, "cudaStreamBeginCapture");
            enqueue_graph_body(b->plan, b->graph_steps, b->capture_stream);
            e = cudaStreamEndCapture(b->capture_stream, &g);
            if (e != cudaSuccess)
                return cuda_fail(b, e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&b->graph_exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess)
                return cuda_fail(b, e, "cudaGraphInstantiate");
        }
        while (left >= b->graph_steps) {
            cudaError_t e = cudaGraphLaunch(b->graph_exec, b->stream);
            if (e != cudaSuccess)
                return cuda_fail(b, e, "cudaGraphLaunch");
            left -= b->graph_steps;
            for (sdm_ctx *c : b->ctxs) {
                c->step += b->graph_steps;
                c->dev_base += b->graph_steps;
            }
        }
    }
    const int64_t off0 = b->ctxs[0]->step - b->ctxs[0]->dev_base;
    enqueue_steps(b->plan, off0, left, b->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_fail(b, e, "step launch");
    for (sdm_ctx *c : b->ctxs)
        c->step += left;
    return SDM_OK;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

sdm_status check_config(const sdm_config *cfg, std::string *err)
{
    if (!cfg)
        return fail(err, SDM_EINVAL, "config is NULL");
    if (cfg->kernel != SDM_KERNEL_GOLOVIN && cfg->kernel != SDM_KERNEL_GEOMETRIC && cfg->kernel != SDM_KERNEL_LONG)
        return fail(err, SDM_EINVAL, "unknown kernel %d", cfg->kernel);
    if (cfg->precision != SDM_PREC_FP64 && cfg->precision != SDM_PREC_KFP32)
        return fail(err, SDM_EINVAL, "unknown precision %d", cfg->precision);
    if (!(std::isfinite(cfg->golovin_b) && cfg->golovin_b >= 0.0 && cfg->golovin_b <= 1e30))
        return fail(err, SDM_EINVAL, "golovin_b must be finite and in [0, 1e30]");
    if (!finite_pos(cfg->dt) || !finite_pos(cfg->dv))
        return fail(err, SDM_EINVAL, "dt and dv must be finite and > 0");
    if (!finite_pos(cfg->ry_k1) || !finite_pos(cfg->ry_k2) || !finite_pos(cfg->ry_k3) || !finite_pos(cfg->ry_r1) ||
        !(cfg->ry_r2 > cfg->ry_r1) || !std::isfinite(cfg->ry_r2))
        return fail(err, SDM_EINVAL, "Rogers-Yau coefficients must be finite, > 0, r1 < r2");
    if (cfg->n_cells < 1)
        return fail(err, SDM_EINVAL, "n_cells must be >= 1");
    if (cfg->cell_base < 0 || (int64_t)cfg->cell_base + cfg->n_cells > INT32_MAX)
        return fail(err, SDM_EINVAL, "cell_base = %d: cell_base + n_cells must lie in [0, 2^31)", cfg->cell_base);
    if (cfg->step0 < 0)
        return fail(err, SDM_EINVAL, "step0 must be >= 0");
    if ((cfg->alloc == nullptr) != (cfg->free == nullptr))
        return fail(err, SDM_EINVAL, "alloc and free must be given together");
    return SDM_OK;
}

// The pre-filter's constants (pair_prefilter_zero), rounded up to binary32
// with a 2^-20 pad: Golovin 2 b; geometric C1 = 4 pi k1 (3 / (4 pi))^(4/3),
// 3 k2, C3 = 4 pi k3 (3 / (4 pi))^(5/6).  The regime volumes 4/3 pi r^3,
// rounded down.
void set_prefilter(InstDev &d)
{
    const double pi = 3.141592653589793;
    auto up = [](double x) { return std::nextafter((float)(x * (1.0 + 0x1p-20)), INFINITY); };
    auto down = [](double x) { return std::nextafter((float)(x * (1.0 - 0x1p-20)), 0.0f); };
    if (d.kernel == SDM_KERNEL_GOLOVIN) {
        d.pre_c[0] = up(2.0 * d.b);
        d.pre_c[1] = d.pre_c[2] = d.pre_c[0];
    } else {
        // Long's efficiency never exceeds c1 R_lim^2 = 1.125
        const double e = d.kernel == SDM_KERNEL_LONG ? 1.125 : 1.0;
        d.pre_c[0] = up(4.0 * pi * d.k1 * std::pow(0.75 / pi, 4.0 / 3.0) * e);
        d.pre_c[1] = up(3.0 * d.k2 * e);
        d.pre_c[2] = up(4.0 * pi * d.k3 * std::pow(0.75 / pi, 5.0 / 6.0) * e);
    }
    d.pre_v[0] = down(4.0 / 3.0 * pi * d.r1 * d.r1 * d.r1);
    d.pre_v[1] = down(4.0 / 3.0 * pi * d.r2 * d.r2 * d.r2);
}

InstDev make_inst(const sdm_ctx *c)
{
    InstDev d{};
    d.xi = c->d_xi;
    d.v = c->d_v;
    d.cell_off = c->d_cell_off;
    d.seed = c->cfg.seed;
    d.step = c->step;
    d.dtdv = c->cfg.dt / c->cfg.dv;
    d.b = c->cfg.golovin_b;
    d.k1 = c->cfg.ry_k1;
    d.k2 = c->cfg.ry_k2;
    d.k3 = c->cfg.ry_k3;
    d.r1 = c->cfg.ry_r1;
    d.r2 = c->cfg.ry_r2;
    d.bf = (float)d.b;
    d.k1f = (float)d.k1;
    d.k2f = (float)d.k2;
    d.k3f = (float)d.k3;
    d.r1f = (float)d.r1;
    d.r2f = (float)d.r2;
    d.dtdvf = (float)d.dtdv;
    d.kernel = c->cfg.kernel;
    d.precision = c->cfg.precision;
    d.n_cells = c->cfg.n_cells;
    set_prefilter(d);
    return d;
}

// Reads the run's device status word (after the stream has been synchronised).
sdm_status check_device_status(sdm_ctx *ctx)
{
    uint32_t status = 0;
    cudaError_t e = cudaMemcpy(&status, &ctx->d_inst->status, sizeof status, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(ctx, e, "status read");
    if (status & 1u)
        return fail(&ctx->error, SDM_ETIMEOUT, "a device-side wait for a bulk copy gave up; results are incomplete");
    if (status & 2u)
        return fail(&ctx->error, SDM_ESTATE,
                    "a sort bucket of a mid-size cell outgrew its room (more than 2048 of the cell's keys in one "
                    "bucket): that cell was not stepped; results are incomplete");
    return SDM_OK;
}

sdm_status ctx_usable(sdm_ctx *ctx)
{
    if (!ctx)
        return fail(nullptr, SDM_EINVAL, "context is NULL");
    if (ctx->broken)
        return fail(&ctx->error, SDM_ESTATE, "context unusable after a CUDA error");
    return SDM_OK;
}

} // namespace

// ======================================================================= ABI
extern "C" {

void sdm_config_default(sdm_config *cfg)
{
    if (!cfg)
        return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->kernel = SDM_KERNEL_GOLOVIN;
    cfg->precision = SDM_PREC_FP64;
    cfg->golovin_b = 1.5e3;
    cfg->dt = 1.0;
    cfg->dv = 1.0e6;
    cfg->ry_k1 = 1.19e8;
    cfg->ry_k2 = 8.0e3;
    cfg->ry_k3 = 201.0;
    cfg->ry_r1 = 40.0e-6;
    cfg->ry_r2 = 600.0e-6;
    cfg->n_cells = 1;
}

int64_t sdm_footprint_bytes(int64_t capacity_sd, int32_t n_cells, int32_t largest_cell)
{
    const int64_t slots = capacity_sd + n_cells + 1;
    int64_t bytes = slots * (8 + 8 + 4) + ((int64_t)n_cells + 2) * 4 + (int64_t)sizeof(InstDev);
    // small per-call scratch kept between calls, by the context and by its own batch
    bytes += 2 * (int64_t)(DevMem::kKeepBlocks * DevMem::kKeepMax);
    if (largest_cell > current_tuning().smem_max_sd) {
        // big-cell scratch, at most: rank and perm per SD; counts per chunk and bucket;
        // liveness bits per chunk
        const int lb = big_lb(largest_cell);
        const int64_t chunks = (capacity_sd + kBigChunk - 1) / kBigChunk + n_cells;
        bytes += capacity_sd * (4 + 4) + (chunks << lb) * 4 + ((int64_t)n_cells << lb) * 4 + chunks * kLiveWords * 4;
    }
    return bytes;
}

sdm_status sdm_create(const sdm_config *cfg, int64_t capacity_sd, void *cuda_stream, sdm_ctx **out)
{
    NvtxRange nvtx_range("sdm_create");
    if (!out)
        return fail(nullptr, SDM_EINVAL, "out is NULL");
    sdm_status st = check_config(cfg, nullptr);
    if (st != SDM_OK)
        return st;
    if (capacity_sd < 1 || capacity_sd + cfg->n_cells + 1 > (int64_t)INT32_MAX)
        return fail(nullptr, SDM_EINVAL, "capacity_sd must be in [1, 2^31 - 2 - n_cells]");
    sdm_ctx *c = new (std::nothrow) sdm_ctx();
    if (!c)
        return fail(nullptr, SDM_ENOMEM, "host allocation failed");
    c->cfg = *cfg;
    c->stream = (cudaStream_t)cuda_stream;
    c->mem.fn = cfg->alloc;
    c->mem.ffn = cfg->free;
    c->mem.user = cfg->alloc_user;
    c->mem.stream = c->stream;
    c->capacity_sd = capacity_sd;
    c->n_slots_cap = capacity_sd + cfg->n_cells + 1; // every group (cells, outside) padded to even
    c->step = cfg->step0;
    c->d_xi = (int64_t *)c->mem.get(sizeof(int64_t) * c->n_slots_cap);
    c->d_v = (double *)c->mem.get(sizeof(double) * c->n_slots_cap);
    c->d_id_of_slot = (int32_t *)c->mem.get(sizeof(int32_t) * c->n_slots_cap);
    c->d_cell_off = (int32_t *)c->mem.get(sizeof(int32_t) * (cfg->n_cells + 2));
    c->d_inst = (InstDev *)c->mem.get(sizeof(InstDev));
    c->device_bytes = c->n_slots_cap * 20 + (int64_t)(cfg->n_cells + 2) * 4 + (int64_t)sizeof(InstDev);
    if (!c->d_xi || !c->d_v || !c->d_id_of_slot || !c->d_cell_off || !c->d_inst) {
        sdm_destroy(c);
        return fail(nullptr, SDM_ENOMEM, "device allocation of %lld SDs failed", (long long)capacity_sd);
    }
    *out = c;
    return SDM_OK;
}

sdm_status sdm_set_attributes(sdm_ctx *ctx, int64_t n_sd, const int64_t *xi, const double *volume,
                              const int32_t *cell_id, int on_device)
{
    NvtxRange nvtx_range("sdm_set_attributes");
    sdm_status st = ctx_usable(ctx);
    if (st != SDM_OK)
        return st;
    if (n_sd < 1 || n_sd > ctx->capacity_sd)
        return fail(&ctx->error, SDM_EINVAL, "n_sd = %lld outside [1, capacity_sd = %lld]", (long long)n_sd,
                    (long long)ctx->capacity_sd);
    if (!xi || !volume || !cell_id)
        return fail(&ctx->error, SDM_EINVAL, "xi, volume and cell_id are required");
    const int32_t n_cells = ctx->cfg.n_cells;
    cudaStream_t s = ctx->stream;
    DevMem &mem = ctx->mem;
    // staging of host inputs
    const size_t b_xi = sizeof(int64_t) * n_sd, b_v = sizeof(double) * n_sd, b_c = sizeof(int32_t) * n_sd;
    void *stage = nullptr;
    const int64_t *dxi = xi;
    const double *dv = volume;
    const int32_t *dcell = cell_id;
    const size_t b_stage = b_xi + b_v + b_c;
    // SD ranges of the pieces (one piece for device input)
    const int n_in = on_device ? 1 : kInChunks;
    int64_t piece[kInChunks + 1];
    for (int k = 0; k <= n_in; ++k)
        piece[k] = n_sd * k / n_in;
    if (!on_device) {
        stage = mem.get(b_stage);
        if (!stage)
            return fail(&ctx->error, SDM_ENOMEM, "staging allocation failed");
        if (!ctx->cstream) {
            CTX_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking));
            for (cudaEvent_t &ev : ctx->in_ev)
                CTX_CUDA(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        }
        char *p = (char *)stage;
        dxi = (const int64_t *)p;
        dv = (const double *)(p + b_xi);
        dcell = (const int32_t *)(p + b_xi + b_v);
        // the copy stream starts after the stream's earlier work (the staging
        // block is free in that order); piece k's copies, then its event
        CTX_CUDA(ctx, cudaEventRecord(ctx->in_ev[kInChunks], s));
        CTX_CUDA(ctx, cudaStreamWaitEvent(ctx->cstream, ctx->in_ev[kInChunks], 0));
        for (int k = 0; k < n_in; ++k) {
            const int64_t a = piece[k], n = piece[k + 1] - piece[k];
            if (n > 0) {
                CTX_CUDA(ctx, cudaMemcpyAsync((void *)(dxi + a), xi + a, sizeof(int64_t) * n, cudaMemcpyHostToDevice,
                                              ctx->cstream));
                CTX_CUDA(ctx, cudaMemcpyAsync((void *)(dv + a), volume + a, sizeof(double) * n,
                                              cudaMemcpyHostToDevice, ctx->cstream));
                CTX_CUDA(ctx, cudaMemcpyAsync((void *)(dcell + a), cell_id + a, sizeof(int32_t) * n,
                                              cudaMemcpyHostToDevice, ctx->cstream));
            }
            CTX_CUDA(ctx, cudaEventRecord(ctx->in_ev[k], ctx->cstream));
        }
    }
    // counts per group (the cells, then the SDs outside the domain), flags,
    // first bad index
    const int32_t n_groups = n_cells + 1;
    const size_t b_counts = sizeof(uint32_t) * n_groups + 16;
    void *meta = mem.get(b_counts);
    if (!meta) {
        mem.put(stage, b_stage);
        return fail(&ctx->error, SDM_ENOMEM, "allocation failed");
    }
    uint32_t *d_counts = (uint32_t *)meta;
    uint32_t *d_flags = d_counts + n_groups;
    unsigned long long *d_bad = (unsigned long long *)(((uintptr_t)(d_flags + 1) + 7) & ~(uintptr_t)7);
    // d_bad lies inside the 16 spare bytes after the counts
    // page-locked staging: the validation block, then poff and uoff (n_groups
    // + 1 each), then the run's record (64-byte aligned pieces)
    auto a64 = [](size_t x) { return (x + 63) & ~(size_t)63; };
    const size_t p_off = a64(b_counts), p_rec = p_off + a64(sizeof(int32_t) * 2 * (n_groups + 1));
    const size_t b_pin = p_rec + a64(sizeof(InstDev));
    if (ctx->h_pin_bytes < b_pin) {
        if (ctx->h_pin)
            cudaFreeHost(ctx->h_pin);
        ctx->h_pin = nullptr;
        ctx->h_pin_bytes = 0;
        if (cudaHostAlloc((void **)&ctx->h_pin, b_pin, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            ctx->h_pin = nullptr;
            mem.put(meta, b_counts);
            mem.put(stage, b_stage);
            return fail(&ctx->error, SDM_ENOMEM, "page-locked host staging allocation failed");
        }
        ctx->h_pin_bytes = b_pin;
    }
    CTX_CUDA(ctx, cudaMemsetAsync(meta, 0, b_counts, s));
    CTX_CUDA(ctx, cudaMemsetAsync(d_bad, 0xFF, sizeof(unsigned long long), s));
    for (int k = 0; k < n_in; ++k) { // piece k once it has landed (pieces land in order)
        if (!on_device)
            CTX_CUDA(ctx, cudaStreamWaitEvent(s, ctx->in_ev[k], 0));
        if (piece[k + 1] > piece[k])
            validate_count_kernel<<<1216, 256, 0, s>>>(piece[k], piece[k + 1], dxi, dv, dcell, n_cells, d_counts,
                                                        d_flags, d_bad);
    }
    // one copy of the whole block (counts, flags, first bad index)
    CTX_CUDA(ctx, cudaMemcpyAsync(ctx->h_pin, meta, b_counts, cudaMemcpyDeviceToHost, s));
    CTX_CUDA(ctx, cudaStreamSynchronize(s));
    const uint32_t *counts = (const uint32_t *)ctx->h_pin;
    const uint32_t flags = counts[n_groups];
    const unsigned long long bad =
        *(const unsigned long long *)(ctx->h_pin + ((uintptr_t)d_bad - (uintptr_t)meta));
    if (flags & 1u) {
        mem.put(meta, b_counts);
        mem.put(stage, b_stage);
        return fail(&ctx->error, SDM_EINVAL,
                    "SD %llu: need xi >= 0, volume in [1e-30, 1e30] m^3, cell in [-1, %d)", bad, n_cells);
    }
    // padded layout: every group starts at an even slot; the SDs outside the
    // domain follow the last cell
    int32_t *poff = (int32_t *)(ctx->h_pin + p_off);
    int32_t *uoff = poff + (n_groups + 1);
    int64_t ps = 0, us = 0;
    int32_t largest = 0;
    for (int32_t c = 0; c < n_groups; ++c) {
        poff[c] = (int32_t)ps;
        uoff[c] = (int32_t)us;
        ps += (counts[c] + 1) & ~1u;
        us += counts[c];
        if (c < n_cells)
            largest = std::max<int32_t>(largest, (int32_t)counts[c]);
    }
    poff[n_groups] = (int32_t)ps;
    uoff[n_groups] = (int32_t)us;
    // slot positions for unsorted input (stable by id)
    std::vector<int32_t> pos;
    if (flags & 2u) {
        std::vector<int32_t> hcell(n_sd);
        if (on_device) {
            CTX_CUDA(ctx, cudaMemcpyAsync(hcell.data(), cell_id, b_c, cudaMemcpyDeviceToHost, s));
            CTX_CUDA(ctx, cudaStreamSynchronize(s));
        } else {
            std::memcpy(hcell.data(), cell_id, b_c);
        }
        pos.resize(n_sd);
        std::vector<int32_t> fill(poff, poff + n_groups);
        for (int64_t i = 0; i < n_sd; ++i)
            pos[i] = fill[hcell[i] < 0 ? n_cells : hcell[i]]++;
    }
    const size_t b_aux = sizeof(int32_t) * 2 * (n_groups + 1) + (pos.empty() ? 0 : b_c);
    void *aux = mem.get(b_aux);
    if (!aux) {
        mem.put(meta, b_counts);
        mem.put(stage, b_stage);
        return fail(&ctx->error, SDM_ENOMEM, "allocation failed");
    }
    int32_t *d_poff = (int32_t *)aux;
    int32_t *d_uoff = d_poff + (n_groups + 1);
    int32_t *d_pos = pos.empty() ? nullptr : d_uoff + (n_groups + 1);
    // poff and uoff lie back to back in both buffers: one copy
    CTX_CUDA(ctx, cudaMemcpyAsync(d_poff, poff, sizeof(int32_t) * 2 * (n_groups + 1), cudaMemcpyHostToDevice, s));
    if (d_pos)
        CTX_CUDA(ctx, cudaMemcpyAsync(d_pos, pos.data(), b_c, cudaMemcpyHostToDevice, s));
    // a context's own launch plan depends only on the padded layout and the
    // launch tuning: kept when both are unchanged
    std::vector<int32_t> cell_off(poff, poff + n_cells + 1);
    const bool keep_plan = ctx->self_batch && ctx->h_cell_off == cell_off &&
                           same_tuning(ctx->self_batch->plan.tuning, current_tuning());
    ctx->n_sd = n_sd;
    ctx->n_slots = ps;
    ctx->largest_cell = largest;
    ctx->h_cell_off = std::move(cell_off);
    ctx->has_positions = false;
    ctx->layout_version += 1;
    ctx->dev_base = ctx->step;
    InstDev *inst = (InstDev *)(ctx->h_pin + p_rec);
    *inst = make_inst(ctx);
    // The small copies come from the page-locked staging and return at
    // once; the next call writes that staging only after its own
    // synchronisation, which follows these copies on the stream.  The
    // scratch is released in stream order: nothing waits for the kernels.
    CTX_CUDA(ctx, cudaMemcpyAsync(ctx->d_cell_off, poff, sizeof(int32_t) * (n_cells + 1), cudaMemcpyHostToDevice, s));
    CTX_CUDA(ctx, cudaMemcpyAsync(ctx->d_inst, inst, sizeof *inst, cudaMemcpyHostToDevice, s));
    fill_padding_kernel<<<(n_groups + 255) / 256, 256, 0, s>>>(n_groups, d_poff, d_uoff, ctx->d_xi, ctx->d_v,
                                                                ctx->d_id_of_slot);
    scatter_kernel<<<1216, 256, 0, s>>>(n_sd, dxi, dv, dcell, n_cells, d_poff, d_uoff, d_pos, ctx->d_xi, ctx->d_v,
                                        ctx->d_id_of_slot);
    CTX_CUDA(ctx, cudaGetLastError());
    mem.put(aux, b_aux);
    mem.put(meta, b_counts);
    mem.put(stage, b_stage);
    ctx->has_attributes = true;
    if (ctx->self_batch && keep_plan)
        ctx->self_batch->versions[0] = ctx->layout_version;
    if (ctx->self_batch && !keep_plan) {
        batch_release(ctx->self_batch);
        delete ctx->self_batch;
        ctx->self_batch = nullptr;
    }
    return SDM_OK;
}

sdm_status sdm_coalescence_step(sdm_ctx *ctx, int32_t n_steps)
{
    NvtxRange nvtx_range("sdm_coalescence_step");
    sdm_status st = ctx_usable(ctx);
    if (st != SDM_OK)
        return st;
    if (!ctx->has_attributes)
        return fail(&ctx->error, SDM_ESTATE, "sdm_set_attributes has not been called");
    if (n_steps < 0)
        return fail(&ctx->error, SDM_EINVAL, "n_steps < 0");
    if (!ctx->self_batch) {
        sdm_batch *b = new (std::nothrow) sdm_batch();
        if (!b)
            return fail(&ctx->error, SDM_ENOMEM, "host allocation failed");
        sdm_ctx *one[1] = {ctx};
        b->own = ctx;
        st = batch_init(b, one, 1, ctx->stream, 0, 0);
        if (st != SDM_OK) {
            ctx->error = b->error;
            batch_release(b);
            delete b;
            return st;
        }
        ctx->self_batch = b;
    }
    st = batch_step(ctx->self_batch, n_steps);
    if (st != SDM_OK)
        ctx->error = ctx->self_batch->error;
    return st;
}

sdm_status sdm_spectrum(sdm_ctx *ctx, const double *r_edges, int32_t n_edges, int per_cell, double *out,
                        int out_on_device)
{
    NvtxRange nvtx_range("sdm_spectrum");
    sdm_status st = ctx_usable(ctx);
    if (st != SDM_OK)
        return st;
    if (!ctx->has_attributes)
        return fail(&ctx->error, SDM_ESTATE, "sdm_set_attributes has not been called");
    if (!r_edges || !out || n_edges < 2 || n_edges > kMaxEdges)
        return fail(&ctx->error, SDM_EINVAL, "need r_edges, out and 2 <= n_edges <= %d", kMaxEdges);
    for (int32_t i = 0; i + 1 < n_edges; ++i)
        if (!(r_edges[i] > 0.0) || !(r_edges[i + 1] > r_edges[i]) || !std::isfinite(r_edges[i + 1]))
            return fail(&ctx->error, SDM_EINVAL, "r_edges must be finite, > 0 and strictly increasing");
    const int32_t nb = n_edges - 1;
    const int64_t n_out = per_cell ? (int64_t)ctx->cfg.n_cells * nb : nb;
    cudaStream_t s = ctx->stream;
    CTX_CUDA(ctx, configure_kernels());
    // the total over all cells with few bins: the atomic-free kernel
    const bool total = !per_cell && nb <= kSpecTotMaxBins;
    const int grid = dev_grids().spec;
    // edges, then dln[b] = ln e[b+1] - ln e[b] (host logarithms), in one copy
    std::vector<double> host_e(r_edges, r_edges + n_edges);
    for (int32_t b = 0; b < nb; ++b)
        host_e.push_back(std::log(r_edges[b + 1]) - std::log(r_edges[b]));
    const size_t b_edges = sizeof(double) * host_e.size(), b_acc = sizeof(double) * n_out;
    const size_t b_part = total ? sizeof(double) * (size_t)grid * nb : b_acc;
    const size_t b_tmp = b_edges + b_part + b_acc;
    // host result: the edges go out of, and the status word comes back into,
    // page-locked staging (the call synchronises before it returns, so the
    // next call finds the staging free)
    constexpr size_t kSpecPin = sizeof(double) * 2 * kMaxEdges + 64;
    if (!out_on_device && !ctx->h_spec) {
        if (cudaHostAlloc((void **)&ctx->h_spec, kSpecPin, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            ctx->h_spec = nullptr;
            return fail(&ctx->error, SDM_ENOMEM, "page-locked host staging allocation failed");
        }
    }
    char *tmp = (char *)ctx->mem.get(b_tmp);
    if (!tmp)
        return fail(&ctx->error, SDM_ENOMEM, "allocation failed");
    double *d_edges = (double *)tmp;
    const double *d_dln = d_edges + n_edges;
    double *d_acc = (double *)(tmp + b_edges);
    double *d_out = out_on_device ? out : (double *)(tmp + b_edges + b_part);
    const double *src_e = host_e.data();
    if (!out_on_device) {
        std::memcpy(ctx->h_spec, host_e.data(), b_edges);
        src_e = (const double *)ctx->h_spec;
    }
    CTX_CUDA(ctx, cudaMemcpyAsync(d_edges, src_e, b_edges, cudaMemcpyHostToDevice, s));
    const double vol = per_cell ? ctx->cfg.dv : ctx->cfg.dv * (double)ctx->cfg.n_cells;
    if (total) {
        spectrum_total_kernel<<<grid, kSpecTotNT, 0, s>>>(ctx->d_inst, ctx->h_cell_off[ctx->cfg.n_cells], d_edges,
                                                          n_edges, d_acc);
        spectrum_total_finalize_kernel<<<nb, 32, 0, s>>>(d_acc, grid, d_dln, nb, vol, d_out);
    } else {
        CTX_CUDA(ctx, cudaMemsetAsync(d_acc, 0, b_acc, s));
        spectrum_kernel<<<ctx->cfg.n_cells, kSpecNT, 0, s>>>(ctx->d_inst, d_edges, n_edges, per_cell ? 1 : 0, d_acc);
        spectrum_finalize_kernel<<<(unsigned)((n_out + 255) / 256), 256, 0, s>>>(d_acc, d_dln, nb, n_out, vol, d_out);
    }
    CTX_CUDA(ctx, cudaGetLastError());
    if (!out_on_device) {
        uint32_t *h_status = (uint32_t *)(ctx->h_spec + sizeof(double) * 2 * kMaxEdges);
        CTX_CUDA(ctx, cudaMemcpyAsync(out, d_out, b_acc, cudaMemcpyDeviceToHost, s));
        CTX_CUDA(ctx, cudaMemcpyAsync(h_status, &ctx->d_inst->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CTX_CUDA(ctx, cudaStreamSynchronize(s));
        ctx->mem.put(tmp, b_tmp);
        if (*h_status & 1u)
            return fail(&ctx->error, SDM_ETIMEOUT, "a device-side wait for a bulk copy gave up; results are incomplete");
        return SDM_OK;
    }
    ctx->mem.put(tmp, b_tmp);
    return SDM_OK;
}

sdm_status sdm_get_attributes(sdm_ctx *ctx, int64_t *xi, double *volume, int on_device)
{
    NvtxRange nvtx_range("sdm_get_attributes");
    sdm_status st = ctx_usable(ctx);
    if (st != SDM_OK)
        return st;
    if (!ctx->has_attributes)
        return fail(&ctx->error, SDM_ESTATE, "sdm_set_attributes has not been called");
    if (!xi && !volume)
        return SDM_OK;
    cudaStream_t s = ctx->stream;
    const int64_t n = ctx->n_sd;
    if (on_device) {
        gather_kernel<<<1216, 256, 0, s>>>(ctx->n_slots, ctx->d_xi, ctx->d_v, ctx->d_id_of_slot, xi, volume);
        CTX_CUDA(ctx, cudaGetLastError());
        return SDM_OK;
    }
    const size_t bx = sizeof(int64_t) * n, bv = sizeof(double) * n;
    char *tmp = (char *)ctx->mem.get(bx + bv);
    if (!tmp)
        return fail(&ctx->error, SDM_ENOMEM, "allocation failed");
    gather_kernel<<<1216, 256, 0, s>>>(ctx->n_slots, ctx->d_xi, ctx->d_v, ctx->d_id_of_slot,
                                       xi ? (int64_t *)tmp : nullptr, volume ? (double *)(tmp + bx) : nullptr);
    CTX_CUDA(ctx, cudaGetLastError());
    if (xi)
        CTX_CUDA(ctx, cudaMemcpyAsync(xi, tmp, bx, cudaMemcpyDeviceToHost, s));
    if (volume)
        CTX_CUDA(ctx, cudaMemcpyAsync(volume, tmp + bx, bv, cudaMemcpyDeviceToHost, s));
    CTX_CUDA(ctx, cudaStreamSynchronize(s));
    ctx->mem.put(tmp, bx + bv);
    return check_device_status(ctx);
}

sdm_status sdm_get_info(const sdm_ctx *ctx, sdm_info *out)
{
    if (!ctx || !out)
        return fail(nullptr, SDM_EINVAL, "context and out are required");
    out->n_sd = ctx->n_sd;
    out->capacity_sd = ctx->capacity_sd;
    out->step = ctx->step;
    out->device_bytes = ctx->device_bytes + (ctx->self_batch ? ctx->self_batch->plan.bytes : 0);
    out->n_cells = ctx->cfg.n_cells;
    out->largest_cell = ctx->largest_cell;
    return SDM_OK;
}

sdm_status sdm_destroy(sdm_ctx *ctx)
{
    NvtxRange nvtx_range("sdm_destroy");
    if (!ctx)
        return SDM_OK;
    if (ctx->self_batch) {
        batch_release(ctx->self_batch);
        delete ctx->self_batch;
    }
    ctx->mem.put(ctx->d_xi, 0);
    ctx->mem.put(ctx->d_v, 0);
    ctx->mem.put(ctx->d_id_of_slot, 0);
    ctx->mem.put(ctx->d_cell_off, 0);
    ctx->mem.put(ctx->d_inst, 0);
    sed_release(ctx);
    cond_release(ctx);
    ctx->mem.release_kept();
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (ctx->h_plan)
        cudaFreeHost(ctx->h_plan);
    if (ctx->plan_ev)
        cudaEventDestroy(ctx->plan_ev);
    if (ctx->h_pin)
        cudaFreeHost(ctx->h_pin);
    if (ctx->h_spec)
        cudaFreeHost(ctx->h_spec);
    for (cudaEvent_t ev : ctx->in_ev)
        if (ev)
            cudaEventDestroy(ev);
    if (ctx->cstream) {
        cudaStreamSynchronize(ctx->cstream);
        cudaStreamDestroy(ctx->cstream);
    }
    delete ctx;
    if (e != cudaSuccess)
        return fail(nullptr, SDM_ECUDA, "sdm_destroy: %s", cudaGetErrorString(e));
    return SDM_OK;
}

const char *sdm_last_error(const sdm_ctx *ctx)
{
    if (ctx)
        return ctx->error.c_str();
    return g_thread_error.c_str();
}

sdm_status sdm_batch_create(sdm_ctx *const *ctxs, int32_t n_ctx, void *cuda_stream, int32_t use_graph,
                            int32_t graph_steps, sdm_batch **out)
{
    NvtxRange nvtx_range("sdm_batch_create");
    if (!out || !ctxs || n_ctx < 1)
        return fail(nullptr, SDM_EINVAL, "need out, ctxs and n_ctx >= 1");
    sdm_batch *b = new (std::nothrow) sdm_batch();
    if (!b)
        return fail(nullptr, SDM_ENOMEM, "host allocation failed");
    sdm_status st = batch_init(b, ctxs, n_ctx, (cudaStream_t)cuda_stream, use_graph, graph_steps);
    if (st != SDM_OK) {
        g_thread_error = b->error;
        batch_release(b);
        delete b;
        return st;
    }
    *out = b;
    return SDM_OK;
}

sdm_status sdm_batch_step(sdm_batch *batch, int32_t n_steps)
{
    NvtxRange nvtx_range("sdm_batch_step");
    if (!batch)
        return fail(nullptr, SDM_EINVAL, "batch is NULL");
    return batch_step(batch, n_steps);
}

sdm_status sdm_batch_destroy(sdm_batch *batch)
{
    NvtxRange nvtx_range("sdm_batch_destroy");
    if (!batch)
        return SDM_OK;
    batch_release(batch);
    cudaError_t e = cudaStreamSynchronize(batch->stream);
    delete batch;
    if (e != cudaSuccess)
        return fail(nullptr, SDM_ECUDA, "sdm_batch_destroy: %s", cudaGetErrorString(e));
    return SDM_OK;
}

sdm_status sdm_set_tuning(const sdm_tuning *t)
{
    sdm_tuning v = {4096, 512, 2, SDM_FUSE_STEPS_DEFAULT, SDM_MID_MAX_SD_DEFAULT};
    if (t) {
        const bool smem_ok = t->smem_max_sd == 512 || t->smem_max_sd == 1024 || t->smem_max_sd == 2048 ||
                             t->smem_max_sd == 4096;
        const bool warp_ok = t->warp_cell_max == 0 || t->warp_cell_max == 64 || t->warp_cell_max == 128 ||
                             t->warp_cell_max == 256 || t->warp_cell_max == 512;
        const bool wpb_ok = t->warps_per_block == 1 || t->warps_per_block == 2 || t->warps_per_block == 4;
        const bool fuse_ok = t->fuse_steps >= 0 && t->fuse_steps <= 1024;
        const bool mid_ok = t->mid_max_sd == 0 || (t->mid_max_sd >= t->smem_max_sd && t->mid_max_sd <= kMidMaxSd);
        if (!smem_ok || !warp_ok || !wpb_ok || !fuse_ok || !mid_ok || t->warp_cell_max > t->smem_max_sd)
            return fail(nullptr, SDM_EINVAL,
                        "tuning: smem_max_sd in {512,1024,2048,4096}, warp_cell_max in {0,64,128,256,512} and <= "
                        "smem_max_sd, warps_per_block in {1,2,4}, fuse_steps in 0..1024, mid_max_sd 0 or in "
                        "[smem_max_sd, 65536]");
        v = *t;
    }
    std::lock_guard<std::mutex> lock(g_tuning_mutex);
    g_tuning = v;
    return SDM_OK;
}

sdm_status sdm_get_tuning(sdm_tuning *out)
{
    if (!out)
        return fail(nullptr, SDM_EINVAL, "out is NULL");
    *out = current_tuning();
    return SDM_OK;
}

sdm_status sdm_diagnostics(sdm_ctx *ctx, sdm_diag *out)
{
    NvtxRange nvtx_range("sdm_diagnostics");
    sdm_status st = ctx_usable(ctx);
    if (st != SDM_OK)
        return st;
    if (!out)
        return fail(&ctx->error, SDM_EINVAL, "out is NULL");
    if (!ctx->has_attributes)
        return fail(&ctx->error, SDM_ESTATE, "no attributes set");
    const int64_t n_in = ctx->h_cell_off[ctx->cfg.n_cells]; // slots of the cells (not the SDs outside)
    // the grid depends on the size only: the same state gives the same bits
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(1216, (n_in + kDiagNT * 8 - 1) / (kDiagNT * 8)));
    const size_t bytes = sizeof(DiagPart) * ((size_t)blocks + 1);
    DiagPart *d = (DiagPart *)ctx->mem.get(bytes);
    if (!d)
        return fail(&ctx->error, SDM_ENOMEM, "diagnostics scratch allocation failed");
    cudaStream_t s = ctx->stream;
    diag_partial_kernel<<<blocks, kDiagNT, 0, s>>>(ctx->d_inst, n_in, d);
    diag_final_kernel<<<1, kDiagNT, 0, s>>>(d, blocks, d + blocks);
    DiagPart h{};
    CTX_CUDA(ctx, cudaGetLastError());
    CTX_CUDA(ctx, cudaMemcpyAsync(&h, d + blocks, sizeof h, cudaMemcpyDeviceToHost, s));
    CTX_CUDA(ctx, cudaStreamSynchronize(s));
    ctx->mem.put(d, bytes);
    out->live_sd = (int64_t)h.live;
    out->sum_xi_lo = h.xi_lo;
    out->sum_xi_hi = h.xi_hi;
    out->sum_xi_v = h.xv;
    return SDM_OK;
}

sdm_status sdm_selftest_bounded_wait(void *cuda_stream, int64_t max_polls)
{
    NvtxRange nvtx_range("sdm_selftest_bounded_wait");
    if (max_polls < 1 || max_polls > (int64_t)1 << 24)
        return fail(nullptr, SDM_EINVAL, "max_polls = %lld outside [1, 2^24]", (long long)max_polls);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint32_t *d = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&d, sizeof(uint32_t), s);
    if (e != cudaSuccess)
        return fail(nullptr, e == cudaErrorMemoryAllocation ? SDM_ENOMEM : SDM_ECUDA, "self-test allocation: %s",
                    cudaGetErrorString(e));
    uint32_t h = 0;
    selftest_wait_kernel<<<1, 32, 0, s>>>((uint32_t)max_polls, d);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    const cudaError_t ef = cudaFreeAsync(d, s);
    if (e == cudaSuccess)
        e = ef;
    if (e != cudaSuccess)
        return fail(nullptr, SDM_ECUDA, "self-test: %s", cudaGetErrorString(e));
    if (h == 1u)
        return fail(nullptr, SDM_ETIMEOUT, "the bounded wait gave up after %lld polls, as designed",
                    (long long)max_polls);
    return fail(nullptr, SDM_ESTATE, "the self-test barrier completed, which it never should");
}

const char *sdm_batch_last_error(const sdm_batch *batch)
{
    if (batch)
        return batch->error.c_str();
    return g_thread_error.c_str();
}

} // extern "C"

// The allocation-free entry point, after the kernels and helpers it uses.
#include "sdm_sediment.cu"
#include "sdm_condense.cu"
#include "sdm_noalloc.cu"
