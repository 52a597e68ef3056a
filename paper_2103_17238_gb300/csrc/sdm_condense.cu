// Condensation step (sdm_condensation_step in include/sdm.h).
//
// The paper lists condensation among the dynamics of its framework and
// prints no formulae.  Reading: the large-drop limit of the diffusional
// growth law, r dr/dt = s G (Rogers & Yau 1989, ch. 7, curvature and solute
// terms dropped), with each cell's supersaturation s and growth coefficient
// G = 1 / (F_k + F_d) held over the step, so r^2 grows by c = 2 G s dt; an
// evaporating SD stops at the floor radius r_min (or at its own radius when
// that is already below it).  The change of volume is evaluated in binary32
// from the binary32 image of the volume and its binary32 radius, in a form
// without cancellation, and added to the binary64 volume (as the fall
// distance of sedimentation is): per SD
//   x = r^2, x' = max(x + c, min(x, r_min^2)), d = c (or floor - x),
//   dV = k43 (d ((x' + a b) + x)) / (a + b), a = sqrt(x'), b = sqrt(x),
//   v' = v + dV.
// Multiplicities do not change.  The per-cell condensed water sum(xi dV) is
// an optional output.
//
// One step on the device (one warp per work item of up to 256 slots of one
// cell, 16-byte loads of xi and v, the binary32 arithmetic per SD, one
// binary64 add per SD to update v):
//   condense_kernel       the update, and per work item the partial sum of
//                         xi dV (one fused multiply-add per SD, lanes in a
//                         fixed shuffle order);
//   condense_cells_kernel per cell, its items' partials in item order.
// HBM traffic: 16 B read and 8 B written per live SD.
//
// Compiled as part of the library's single translation unit (included at the
// end of sdm_runtime.cu).

namespace {

constexpr int kCondItem = 256; // slots per work item (a multiple of 2: cells start at even slots)
constexpr int kCondNT = 256;
constexpr float kR3ToVolF = (float)(4.0 * kPi / 3.0); // 4 pi / 3 (binary64 pi) rounded to binary32

struct __align__(16) CondItem {
    int32_t cell;
    int32_t begin; // first slot
    int32_t n;     // slots (<= kCondItem), even
    int32_t pad;
};

struct CondBuffers {
    int64_t layout_version = -1; // the layout the work list was built for
    int32_t n_items = 0;
    CondItem *items = nullptr;
    int32_t *item_start = nullptr; // n_cells + 1
    float *cf = nullptr;           // n_cells: c of each cell, binary32
    double *partial = nullptr;     // n_items
    double *cond = nullptr;        // n_cells
    float *h_cf = nullptr;         // page-locked staging of cf
    cudaEvent_t cf_done = nullptr; // the last copy out of h_cf
    std::vector<float> last_cf;    // cf on the device (no copy when a call repeats it)
};

// f2d_exact (sdm_sediment.cu): the exact widening of a binary32 on the
// integer pipe.

// dV of one live SD (the reading above), binary32.  The binary32 image of
// v is rounded on the integer pipe (d2f_rn): the conversion instruction would
// take the narrow binary64 pipe, which then bounds the kernel.
__device__ __forceinline__ float condense_dv(double v, float cf, float xminf)
{
    bool in_range;
    const float r = radius32(d2f_rn(v, in_range)); // volumes lie in [1e-30, 1e30]: always in range
    const float x = __fmul_rn(r, r);
    float xn = __fadd_rn(x, cf);
    const float lo = x < xminf ? x : xminf;
    float d = cf;
    if (xn < lo) {
        xn = lo;
        d = __fsub_rn(lo, x);
    }
    if (d == 0.0f)
        return 0.0f;
    const float a = __fsqrt_rn(xn), b = __fsqrt_rn(x);
    const float num = __fmul_rn(d, __fadd_rn(__fadd_rn(xn, __fmul_rn(a, b)), x));
    return __fmul_rn(kR3ToVolF, __fdiv_rn(num, __fadd_rn(a, b)));
}

__global__ void __launch_bounds__(kCondNT) condense_kernel(const CondItem *__restrict__ items, int32_t n_items,
                                                           const int64_t *__restrict__ xi, double *__restrict__ v,
                                                           const float *__restrict__ cf, float xminf,
                                                           double *__restrict__ partial)
{
    constexpr int PAIRS = kCondItem / 64; // SD pairs per lane
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int it = gw; it < n_items; it += nw) {
        const CondItem I = items[it];
        const float c = cf[I.cell];
        const longlong2 *x2 = reinterpret_cast<const longlong2 *>(xi + I.begin);
        double2 *v2 = reinterpret_cast<double2 *>(v + I.begin);
        const int np = I.n / 2;
        longlong2 xs[PAIRS];
        double2 vs[PAIRS];
#pragma unroll
        for (int k = 0; k < PAIRS; ++k) { // every load of the item first
            const int q = lane + 32 * k;
            if (q < np) {
                xs[k] = x2[q];
                vs[k] = v2[q];
            }
        }
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < PAIRS; ++k) {
            const int q = lane + 32 * k;
            if (q >= np)
                continue;
            double2 w = vs[k];
            bool changed = false;
            if (xs[k].x > 0) {
                const float dv = condense_dv(w.x, c, xminf);
                if (dv != 0.0f) {
                    const double dd = f2d_exact(dv);
                    w.x = __dadd_rn(w.x, dd);
                    if (partial)
                        acc = __fma_rn(xi2d(xs[k].x), dd, acc);
                    changed = true;
                }
            }
            if (xs[k].y > 0) {
                const float dv = condense_dv(w.y, c, xminf);
                if (dv != 0.0f) {
                    const double dd = f2d_exact(dv);
                    w.y = __dadd_rn(w.y, dd);
                    if (partial)
                        acc = __fma_rn(xi2d(xs[k].y), dd, acc);
                    changed = true;
                }
            }
            if (changed)
                v2[q] = w;
        }
        if (partial) {
#pragma unroll
            for (int d = 16; d > 0; d >>= 1)
                acc = __dadd_rn(acc, __shfl_down_sync(0xFFFFFFFFu, acc, d));
            if (lane == 0)
                partial[it] = acc;
        }
    }
}

// condensed[c] = the partial sums of cell c's items (one warp per cell)
__global__ void __launch_bounds__(kCondNT) condense_cells_kernel(const int32_t *__restrict__ item_start,
                                                                 int32_t n_cells, const double *__restrict__ partial,
                                                                 double *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int c = gw; c < n_cells; c += nw) {
        double acc = 0.0;
        for (int i = item_start[c] + lane; i < item_start[c + 1]; i += 32)
            acc = __dadd_rn(acc, partial[i]);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1)
            acc = __dadd_rn(acc, __shfl_down_sync(0xFFFFFFFFu, acc, d));
        if (lane == 0)
            out[c] = acc;
    }
}

void cond_release(sdm_ctx *ctx)
{
    if (!ctx->cond)
        return;
    CondBuffers &b = *ctx->cond;
    void *bufs[] = {b.items, b.item_start, b.cf, b.partial, b.cond};
    for (void *p : bufs)
        ctx->mem.put(p, 0);
    if (b.cf_done) {
        cudaEventSynchronize(b.cf_done);
        cudaEventDestroy(b.cf_done);
    }
    if (b.h_cf)
        cudaFreeHost(b.h_cf);
    delete ctx->cond;
    ctx->cond = nullptr;
}

// The work list of the current layout (rebuilt when the layout changes).
sdm_status cond_prepare(sdm_ctx *ctx)
{
    const int32_t nc = ctx->cfg.n_cells;
    if (!ctx->cond) {
        ctx->cond = new CondBuffers();
        CondBuffers &b = *ctx->cond;
        b.cf = static_cast<float *>(ctx->mem.get(sizeof(float) * nc));
        b.cond = static_cast<double *>(ctx->mem.get(sizeof(double) * nc));
        b.item_start = static_cast<int32_t *>(ctx->mem.get(sizeof(int32_t) * (nc + 1)));
        if (!b.cf || !b.cond || !b.item_start) {
            cond_release(ctx);
            return fail(&ctx->error, SDM_ENOMEM, "condensation: device allocation failed");
        }
        cudaError_t e = cudaMallocHost(&b.h_cf, sizeof(float) * nc);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&b.cf_done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cond_release(ctx);
            return fail(&ctx->error, SDM_ENOMEM, "condensation: page-locked staging failed");
        }
    }
    CondBuffers &b = *ctx->cond;
    if (b.layout_version == ctx->layout_version)
        return SDM_OK;
    std::vector<CondItem> items;
    std::vector<int32_t> start(nc + 1);
    for (int32_t c = 0; c < nc; ++c) {
        start[c] = (int32_t)items.size();
        const int32_t lo = ctx->h_cell_off[c], hi = ctx->h_cell_off[c + 1];
        for (int32_t o = lo; o < hi; o += kCondItem)
            items.push_back(CondItem{c, o, std::min(kCondItem, hi - o), 0});
    }
    start[nc] = (int32_t)items.size();
    ctx->mem.put(b.items, 0);
    ctx->mem.put(b.partial, 0);
    b.items = nullptr;
    b.partial = nullptr;
    b.n_items = (int32_t)items.size();
    b.layout_version = -1;
    const size_t ni = std::max<size_t>(1, items.size());
    b.items = static_cast<CondItem *>(ctx->mem.get(sizeof(CondItem) * ni));
    b.partial = static_cast<double *>(ctx->mem.get(sizeof(double) * ni));
    if (!b.items || !b.partial)
        return fail(&ctx->error, SDM_ENOMEM, "condensation: device allocation failed");
    cudaStream_t s = ctx->stream;
    CTX_CUDA(ctx, cudaMemcpyAsync(b.items, items.data(), sizeof(CondItem) * items.size(), cudaMemcpyHostToDevice, s));
    CTX_CUDA(ctx, cudaMemcpyAsync(b.item_start, start.data(), sizeof(int32_t) * (nc + 1), cudaMemcpyHostToDevice, s));
    // the host vectors go out of scope: wait for the copies of pageable memory
    CTX_CUDA(ctx, cudaStreamSynchronize(s));
    b.layout_version = ctx->layout_version;
    return SDM_OK;
}

} // namespace

extern "C" sdm_status sdm_condensation_step(sdm_ctx *ctx, const double *G, const double *s, double r_min,
                                            double *condensed, int condensed_on_device)
{
    NvtxRange nvtx_range("sdm_condensation_step");
    sdm_status st = ctx_usable(ctx);
    if (st != SDM_OK)
        return st;
    if (!ctx->has_attributes)
        return fail(&ctx->error, SDM_ESTATE, "sdm_set_attributes has not been called");
    if (!G || !s)
        return fail(&ctx->error, SDM_EINVAL, "G and s (one value per cell) are required");
    if (!(r_min >= 1e-9 && r_min <= 1e-3))
        return fail(&ctx->error, SDM_EINVAL, "r_min = %g outside [1e-9, 1e-3] m", r_min);
    const int32_t nc = ctx->cfg.n_cells;
    const double dt = ctx->cfg.dt;
    for (int32_t c = 0; c < nc; ++c) {
        if (!(std::isfinite(G[c]) && G[c] >= 0.0) || !(std::isfinite(s[c]) && s[c] >= -1.0 && s[c] <= 1.0))
            return fail(&ctx->error, SDM_EINVAL, "cell %d: G = %g must be finite and >= 0, s = %g in [-1, 1]", c, G[c],
                        s[c]);
        if (!(std::fabs(((2.0 * G[c]) * s[c]) * dt) <= 1e-6))
            return fail(&ctx->error, SDM_EINVAL, "cell %d: |2 G s dt| = %g m^2 above 1e-6 m^2", c,
                        std::fabs(((2.0 * G[c]) * s[c]) * dt));
    }
    st = cond_prepare(ctx);
    if (st != SDM_OK)
        return st;
    CondBuffers &b = *ctx->cond;
    cudaStream_t cs = ctx->stream;
    std::vector<float> cf(nc);
    for (int32_t c = 0; c < nc; ++c)
        cf[c] = (float)(((2.0 * G[c]) * s[c]) * dt);
    if (cf != b.last_cf) { // a new field (a repeated one is on the device already)
        CTX_CUDA(ctx, cudaEventSynchronize(b.cf_done)); // the staging's last copy has left
        std::memcpy(b.h_cf, cf.data(), sizeof(float) * nc);
        CTX_CUDA(ctx, cudaMemcpyAsync(b.cf, b.h_cf, sizeof(float) * nc, cudaMemcpyHostToDevice, cs));
        CTX_CUDA(ctx, cudaEventRecord(b.cf_done, cs));
        b.last_cf.swap(cf);
    }
    const float xminf = (float)(r_min * r_min);
    if (b.n_items > 0) {
        const int grid = (int)std::min<int64_t>((b.n_items + kCondNT / 32 - 1) / (kCondNT / 32), 152 * 8);
        condense_kernel<<<grid, kCondNT, 0, cs>>>(b.items, b.n_items, ctx->d_xi, ctx->d_v, b.cf, xminf,
                                                  condensed ? b.partial : nullptr);
    }
    if (condensed) {
        const int grid = (int)std::min<int64_t>((nc + kCondNT / 32 - 1) / (kCondNT / 32), 152 * 8);
        condense_cells_kernel<<<grid, kCondNT, 0, cs>>>(b.item_start, nc, b.partial, b.cond);
    }
    CTX_CUDA(ctx, cudaGetLastError());
    if (condensed) {
        if (condensed_on_device) {
            CTX_CUDA(ctx, cudaMemcpyAsync(condensed, b.cond, sizeof(double) * nc, cudaMemcpyDeviceToDevice, cs));
        } else {
            CTX_CUDA(ctx, cudaMemcpyAsync(condensed, b.cond, sizeof(double) * nc, cudaMemcpyDeviceToHost, cs));
            CTX_CUDA(ctx, cudaStreamSynchronize(cs));
        }
    }
    return SDM_OK;
}
