// Allocation-free coalescence step of one cell held in caller-owned device
// arrays (sdm_cell_step_noalloc in include/sdm.h).
//
// Some callers cannot allocate device memory while they run: a host model
// that reserves all of its GPU memory up front in its own pool and forbids
// allocation afterwards, a Fortran/OpenACC code whose runtime owns every
// device buffer, a latency-bound loop that cannot afford an allocator call.
// This entry point serves them: the caller passes the cell's arrays, and the
// large-cell kernels' scratch (sort keys, ranks, permutation, bucket counts)
// together with their work lists and run record live in one fixed-size,
// file-scope device array, set up once per device.
//
// Compiled as part of the library's single translation unit (included at the
// end of sdm_runtime.cu), after the kernels it launches.

#include <initializer_list>
#include <mutex>

namespace {

constexpr int64_t kNaMaxSd = SDM_NOALLOC_MAX_SD;
constexpr int kNaMaxLb = 10; // buckets for kNaMaxSd SDs (2^20 / 1024)
constexpr int64_t kNaMaxChunks = (kNaMaxSd + kBigChunk - 1) / kBigChunk;
constexpr int64_t kNaMaxPairBlocks = ((kNaMaxSd / 2 + 1) / 2 + kPairNT - 1) / kPairNT;

constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of the pieces inside the array.
constexpr size_t kNaRank = 0;
constexpr size_t kNaPerm = na_align(kNaRank + 4 * (size_t)kNaMaxSd);
constexpr size_t kNaHist = na_align(kNaPerm + 4 * (size_t)kNaMaxSd);
constexpr size_t kNaBstart = na_align(kNaHist + 4 * (size_t)kNaMaxChunks * ((size_t)1 << kNaMaxLb));
constexpr size_t kNaScale = na_align(kNaBstart + 4 * (((size_t)1 << kNaMaxLb) + 1));
constexpr size_t kNaScaleF = na_align(kNaScale + 8);
constexpr size_t kNaBig = na_align(kNaScaleF + 4);
constexpr size_t kNaChunks = na_align(kNaBig + sizeof(BigCell));
constexpr size_t kNaBuckets = na_align(kNaChunks + sizeof(BigChunk) * (size_t)kNaMaxChunks);
constexpr size_t kNaPairs = na_align(kNaBuckets + sizeof(BigBucket) * ((size_t)1 << kNaMaxLb));
constexpr size_t kNaInst = na_align(kNaPairs + sizeof(BigPairs) * (size_t)kNaMaxPairBlocks);
constexpr size_t kNaInsts = na_align(kNaInst + sizeof(InstDev));
constexpr size_t kNaCellOff = na_align(kNaInsts + sizeof(InstDev *));
constexpr size_t kNaBytes = na_align(kNaCellOff + 2 * sizeof(int32_t));

// About 8.6 MiB; every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Fills the run record, the one-cell descriptor and the work lists in the
// array (nothing has to start at zero beyond what is written here; the
// kernels overwrite every count and position they read).
__global__ void noalloc_setup_kernel(unsigned char *base, InstDev inst, int32_t n, int32_t lb, int32_t n_chunks,
                                     int32_t n_pair_blocks)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    if (gid == 0) {
        int32_t *cell_off = reinterpret_cast<int32_t *>(base + kNaCellOff);
        cell_off[0] = 0;
        cell_off[1] = n;
        InstDev *rec = reinterpret_cast<InstDev *>(base + kNaInst);
        inst.cell_off = cell_off;
        inst.status = 0;
        *rec = inst;
        *reinterpret_cast<InstDev **>(base + kNaInsts) = rec;
        BigCell bc{};
        bc.inst = 0;
        bc.cell = 0;
        bc.n = n;
        bc.lb = lb;
        bc.n_chunks = n_chunks;
        *reinterpret_cast<BigCell *>(base + kNaBig) = bc;
    }
    BigChunk *chunks = reinterpret_cast<BigChunk *>(base + kNaChunks);
    BigBucket *buckets = reinterpret_cast<BigBucket *>(base + kNaBuckets);
    BigPairs *pairs = reinterpret_cast<BigPairs *>(base + kNaPairs);
    for (int i = gid; i < n_chunks; i += stride)
        chunks[i] = BigChunk{0, i};
    for (int i = gid; i < (1 << lb); i += stride)
        buckets[i] = BigBucket{0, i};
    for (int i = gid; i < n_pair_blocks; i += stride)
        pairs[i] = BigPairs{0, i * kPairNT};
}

std::mutex g_na_mutex;
unsigned char *g_na_base[64] = {};

// Per-device set-up, with that device current: the array's device address
// (host code only sees a stand-in symbol) and the kernels' shared-memory
// limits.  Done by the first call on each device.
sdm_status noalloc_base(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fail(nullptr, SDM_ECUDA, "sdm_cell_step_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 64)
        return fail(nullptr, SDM_EINVAL, "sdm_cell_step_noalloc: device ordinal %d above 63", dev);
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_base[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(nullptr, SDM_ECUDA, "sdm_cell_step_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        const int hb = (int)big_hist_smem(kBigMaxLB);
        if ((e = cudaFuncSetAttribute(big_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, hb)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(big_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, hb)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(big_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, hb)) != cudaSuccess)
            return fail(nullptr, SDM_ECUDA, "sdm_cell_step_noalloc: kernel set-up: %s", cudaGetErrorString(e));
        g_na_base[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_na_base[dev];
    return SDM_OK;
}

} // namespace

extern "C" sdm_status sdm_cell_step_noalloc(const sdm_config *cfg, int64_t step, int64_t *xi, double *volume,
                                            int64_t n_sd, void *cuda_stream)
{
    NvtxRange nvtx_range("sdm_cell_step_noalloc");
    sdm_status st = check_config(cfg, nullptr);
    if (st != SDM_OK)
        return st;
    if (cfg->n_cells != 1 || cfg->cell_base != 0)
        return fail(nullptr, SDM_EINVAL,
                    "sdm_cell_step_noalloc: cfg->n_cells must be 1 and cfg->cell_base 0 (one cell per call, random "
                    "streams of cell index 0)");
    if (step < 0)
        return fail(nullptr, SDM_EINVAL, "sdm_cell_step_noalloc: step must be >= 0");
    if (n_sd < 2 || n_sd > kNaMaxSd || (n_sd & 1))
        return fail(nullptr, SDM_EINVAL,
                    "sdm_cell_step_noalloc: n_sd = %lld must be even and in [2, %lld] (SDM_NOALLOC_MAX_SD); "
                    "pad an odd cell with one dead SD (xi = 0)",
                    (long long)n_sd, (long long)kNaMaxSd);
    if (!xi || !volume || ((uintptr_t)xi & 15) || ((uintptr_t)volume & 15))
        return fail(nullptr, SDM_EINVAL, "sdm_cell_step_noalloc: xi and volume must be 16-byte aligned device arrays");
    // an error left by earlier, unrelated work on this thread is reported as
    // such and left in place for its owner (the final check below would
    // otherwise take it for this call's launch failure and clear it)
    cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess)
        return fail(nullptr, SDM_ECUDA, "sdm_cell_step_noalloc: a CUDA error from earlier work is pending: %s",
                    cudaGetErrorString(pending));
    unsigned char *base = nullptr;
    st = noalloc_base(&base);
    if (st != SDM_OK)
        return st;
    // both arrays must be memory of the current device (a host pointer or
    // another device's buffer would fault inside the kernels); the query
    // allocates nothing
    int cur = 0;
    cudaGetDevice(&cur);
    for (const void *ptr : {(const void *)xi, (const void *)volume}) {
        cudaPointerAttributes a{};
        const cudaError_t pe = cudaPointerGetAttributes(&a, ptr);
        if (pe != cudaSuccess) {
            cudaGetLastError(); // the query's own error, not a launch failure
            return fail(nullptr, SDM_EINVAL, "sdm_cell_step_noalloc: pointer query failed: %s",
                        cudaGetErrorString(pe));
        }
        if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != cur)
            return fail(nullptr, SDM_EINVAL,
                        "sdm_cell_step_noalloc: xi and volume must be device (or managed) memory of the current "
                        "device %d",
                        cur);
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    InstDev inst{};
    inst.xi = xi;
    inst.v = volume;
    inst.seed = cfg->seed;
    inst.step = step;
    inst.dtdv = cfg->dt / cfg->dv;
    inst.b = cfg->golovin_b;
    inst.k1 = cfg->ry_k1;
    inst.k2 = cfg->ry_k2;
    inst.k3 = cfg->ry_k3;
    inst.r1 = cfg->ry_r1;
    inst.r2 = cfg->ry_r2;
    inst.bf = (float)inst.b;
    inst.k1f = (float)inst.k1;
    inst.k2f = (float)inst.k2;
    inst.k3f = (float)inst.k3;
    inst.r1f = (float)inst.r1;
    inst.r2f = (float)inst.r2;
    inst.dtdvf = (float)inst.dtdv;
    inst.kernel = cfg->kernel;
    set_prefilter(inst);
    inst.precision = cfg->precision;
    inst.n_cells = 1;
    const int n = (int)n_sd;
    const int lb = big_lb(n);
    if (lb > kNaMaxLb) // cannot happen for n <= kNaMaxSd; the tables are sized for kNaMaxLb
        return fail(nullptr, SDM_EINVAL, "sdm_cell_step_noalloc: %d buckets exceed the static tables", 1 << lb);
    const int n_chunks = (n + kBigChunk - 1) / kBigChunk;
    const int n_pair_blocks = ((n / 2 + 1) / 2 + kPairNT - 1) / kPairNT;
    noalloc_setup_kernel<<<16, 256, 0, s>>>(base, inst, n, lb, n_chunks, n_pair_blocks);
    BigScratch S;
    S.hist = reinterpret_cast<uint32_t *>(base + kNaHist);
    S.bstart = reinterpret_cast<uint32_t *>(base + kNaBstart);
    S.rank = reinterpret_cast<uint32_t *>(base + kNaRank);
    S.perm = reinterpret_cast<uint32_t *>(base + kNaPerm);
    S.scale = reinterpret_cast<double *>(base + kNaScale);
    S.scale_f = reinterpret_cast<float *>(base + kNaScaleF);
    const BigCell *big = reinterpret_cast<const BigCell *>(base + kNaBig);
    const BigChunk *chunks = reinterpret_cast<const BigChunk *>(base + kNaChunks);
    const BigBucket *buckets = reinterpret_cast<const BigBucket *>(base + kNaBuckets);
    const BigPairs *pairs = reinterpret_cast<const BigPairs *>(base + kNaPairs);
    InstDev *const *insts = reinterpret_cast<InstDev *const *>(base + kNaInsts);
    const size_t hs = big_hist_smem(lb);
    big_hist_kernel<<<n_chunks, kBigNT, hs, s>>>(chunks, big, insts, S, 0);
    const int tiles = std::max(1, (1 << lb) / kBigColNT);
    big_colscan_kernel<<<tiles, kBigColNT, 0, s>>>(big, tiles, S);
    big_scan_kernel<<<1, kBigNT, big_hist_smem(kBigMaxLB), s>>>(big, insts, S);
    big_scatter_kernel<<<n_chunks, kBigNT, hs, s>>>(chunks, big, insts, S, 0);
    big_bucket_sort_kernel<<<1 << lb, kBucketNT, 0, s>>>(buckets, big, insts, S, 0);
    big_pairs_kernel<<<n_pair_blocks, kPairNT, 0, s>>>(pairs, big, insts, S, 0);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(nullptr, SDM_ECUDA, "sdm_cell_step_noalloc: launch: %s", cudaGetErrorString(e));
    return SDM_OK;
}
