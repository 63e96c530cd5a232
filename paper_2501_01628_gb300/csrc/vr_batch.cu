// vr_batch.cu -- the batched form: many renders (volumes x views) and all their
// compositing in one persistent, cooperative, CUDA-graph-captured launch.
//
// Sec. 4 of arXiv:2501.01628 renders time-varying data with several fields,
// several parts per GPU, interactively; Sec. 2.2 notes that data-parallel
// rendering combines with replication (here: many views of resident data). Work
// items are claimed from one atomic counter in render-major order: the (brick,
// tile) march items of render r, then its composite tiles. A composite tile
// waits until every march item of its render has finished; a march item waits
// until the partial-image ring slot it reuses has been composited. Every item
// waited on was claimed earlier by a block that is already running, so waits
// always end; each is still bounded, and a wait that gives up sets an error bit
// (vr_sync reports VR_ERR_TIMEOUT) instead of hanging.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "vr_device.cuh"
#include "vr_objects.h"

namespace vr {
namespace {

// Bounded wait for *addr >= target. Gives up after `limit` sleeps, or at once
// when another block has already given up (the error word is set), so one
// failed wait cannot turn into a long series of timeouts.
__device__ __forceinline__ bool wait_at_least(const int *addr, int target, int limit, const int *error)
{
    const volatile int *a = addr;
    const volatile int *err = error;
    for (int i = 0; i < limit; ++i) {
        if (*a >= target) {
            __threadfence();
            return true;
        }
        if (*err & 2) return false;
        __nanosleep(128);
    }
    return false;
}

template <typename S, bool OPC>
__global__ void __launch_bounds__(128, 9) batch_kernel(const __grid_constant__ BatchParams p)
{
    __shared__ long long s_item;
    __shared__ int s_brick[kMaxBricks];
    __shared__ int s_m;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ph = 32 / p.pw, tw = 2 * p.pw, th = 2 * ph;
    for (;;) {
        if (tid == 0) {
            const volatile int *err = p.error;
            // stop claiming once any wait has given up: remaining items are skipped
            s_item = (*err & 2) ? p.total_items : static_cast<long long>(atomicAdd(p.claim, 1ULL));
        }
        __syncthreads();
        const long long item = s_item;
        __syncthreads();
        if (item >= p.total_items) break;
        // segment g holds the march items of unit g, then the composite tiles of
        // unit g-1 (composited one unit late, so they rarely wait). A unit is one
        // render (render-major order) or one volume with all its views, its
        // march items ordered brick by brick (brick-major order: a brick's data
        // stays in L2 while every view marches it).
        int lo = 0, hi = p.n_units;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.render_begin[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const int g = lo;
        int local = static_cast<int>(item - p.render_begin[g]);
        const int gm = g < p.n_units ? p.unit_march[g] : 0;
        const bool is_march = local < gm;
        if (!is_march) local -= gm;
        const int u = is_march ? g : g - 1;
        float4 *slot = p.ring + static_cast<long long>(u % p.slots) * p.slot_px;
        if (is_march) {
            // the ring slot must have been composited by the unit that used it last
            if (tid == 0 && u >= p.slots) {
                const int pu = u - p.slots;
                if (!wait_at_least(p.comp_done + pu, p.unit_comp[pu], p.wait_limit, p.error)) atomicOr(p.error, 2);
            }
            __syncthreads();
            int w, v, t;
            const BrickLaunch *Bp;
            if (p.mode == 0) {
                w = u % p.n_views;
                v = u / p.n_views;
                const BrickLaunch *vb = p.vb + static_cast<long long>(w) * p.nb;
                int blo = 0, bhi = p.nb - 1;
                while (blo < bhi) {
                    const int mid = (blo + bhi + 1) >> 1;
                    if (vb[mid].item_begin <= local) blo = mid;
                    else bhi = mid - 1;
                }
                Bp = vb + blo;
                t = local - Bp->item_begin;
            } else {
                v = u;
                int klo = 0, khi = p.nb * p.n_views - 1;
                while (klo < khi) {
                    const int mid = (klo + khi + 1) >> 1;
                    if (p.bw_begin[mid] <= local) klo = mid;
                    else khi = mid - 1;
                }
                const int bb = klo / p.n_views;
                w = klo - bb * p.n_views;
                Bp = p.vb + static_cast<long long>(w) * p.nb + bb;
                t = local - static_cast<int>(p.bw_begin[klo]);
            }
            const BrickLaunch &B = *Bp;
            const BatchView &V = p.views[w];
            float4 *part = slot + static_cast<long long>(w) * p.view_stride;
            const int ty = t / B.tiles_x, tx = t - ty * B.tiles_x;
            const int rx = tx * tw + (warp & 1) * p.pw + lane % p.pw;
            const int ry = ty * th + (warp >> 1) * ph + lane / p.pw;
            if (rx < B.rect[2] && ry < B.rect[3]) {
                dev::OwnedRun run;
                dev::owned_run(V, B, B.rect[0] + rx, B.rect[1] + ry, run);
                unsigned long long unused = 0;
                const float2 sb = p.vol_tf[v];
                part[B.poff + static_cast<long long>(ry) * B.rect[2] + rx] =
                    dev::march_run<S, false, OPC>(p.vol_data[v], B, run, p.tf, sb.x, sb.y, p.ntf, p.ert_T, unused,
                                                  p.opc_ratio);
            }
            __threadfence();  // every writer publishes its partial before the count moves
            __syncthreads();
            if (tid == 0) atomicAdd(p.march_done + u, 1);
        } else {
            int w, r, c = local;
            if (p.mode == 0) {
                w = u % p.n_views;
                r = u;
            } else {
                const int per_view = p.views[0].comp_items;  // every view has the same image size
                w = c / per_view;
                c -= w * per_view;
                r = u * p.n_views + w;
            }
            const BatchView &V = p.views[w];
            const float4 *part = slot + static_cast<long long>(w) * p.view_stride;
            const int ntx = (V.W + kBatchCompW - 1) / kBatchCompW;
            const int cty = c / ntx, ctx = c - cty * ntx;
            const int tx0 = ctx * kBatchCompW, ty0 = cty * kBatchCompH;
            // (wait_extra raises unit 0's target past its item count: a test hook
            // that makes this bounded wait give up; 0 in normal use)
            if (tid == 0 && !wait_at_least(p.march_done + u, p.unit_march[u] + (u == 0 ? p.wait_extra : 0),
                                           p.wait_limit, p.error))
                atomicOr(p.error, 2);
            __syncthreads();
            const BrickLaunch *vb = p.vb + static_cast<long long>(w) * p.nb;
            const int *order = p.order + static_cast<long long>(w) * p.nb;
            if (warp == 0) {
                int m = 0;
                for (int j0 = 0; j0 < p.nb; j0 += 32) {
                    const int j = j0 + lane;
                    bool ov = false;
                    int b = 0;
                    if (j < p.nb) {
                        b = order[j];
                        const int *rc = vb[b].rect;
                        ov = rc[0] < tx0 + kBatchCompW && tx0 < rc[0] + rc[2] && rc[1] < ty0 + kBatchCompH &&
                             ty0 < rc[1] + rc[3];
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, ov);
                    if (ov) s_brick[m + __popc(bal & ((1u << lane) - 1u))] = b;
                    m += __popc(bal);
                }
                if (lane == 0) s_m = m;
            }
            __syncthreads();
            const int px = tx0 + (tid % kBatchCompW), py = ty0 + tid / kBatchCompW;
            if (px < V.W && py < V.H) {
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                const int m = s_m;
                for (int i = 0; i < m; ++i) {
                    const BrickLaunch &B = vb[s_brick[i]];
                    const int x0 = B.rect[0], y0 = B.rect[1], bw = B.rect[2], bh = B.rect[3];
                    if (px >= x0 && px < x0 + bw && py >= y0 && py < y0 + bh)
                        acc = dev::over(acc, part[B.poff + static_cast<long long>(py - y0) * bw + (px - x0)]);
                }
                p.out[(static_cast<long long>(r) * V.H + py) * V.W + px] = acc;
            }
            __threadfence();
            __syncthreads();  // every read of the ring slot is done before it is released
            if (tid == 0) atomicAdd(p.comp_done + u, 1);
        }
    }
}

template <typename S, bool OPC>
cudaError_t launch_batch_t(const BatchParams &p, int blocks, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_kernel<S, OPC>, p);
}

}  // namespace

template <typename S>
cudaError_t launch_batch_s(const BatchParams &p, int blocks, cudaStream_t s)
{
    return p.opc_ratio != 1.0f ? launch_batch_t<S, true>(p, blocks, s) : launch_batch_t<S, false>(p, blocks, s);
}

cudaError_t launch_batch(const BatchParams &p, int kind, int blocks, cudaStream_t s)
{
    switch (kind) {
    case kStoreF32: return launch_batch_s<float>(p, blocks, s);
    case kStoreBF16: return launch_batch_s<__nv_bfloat16>(p, blocks, s);
    case kStoreF16: return launch_batch_s<__half>(p, blocks, s);
    case kStoreBF16Oct: return launch_batch_s<dev::Octet<__nv_bfloat16>>(p, blocks, s);
    case kStoreF16Oct: return launch_batch_s<dev::Octet<__half>>(p, blocks, s);
    default: return cudaErrorInvalidValue;
    }
}

int batch_max_blocks_per_sm(int kind)
{
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (kind) {
    case kStoreF32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<float, true>, 128, 0); break;
    case kStoreBF16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<__nv_bfloat16, true>, 128, 0); break;
    case kStoreF16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<__half, true>, 128, 0); break;
    case kStoreBF16Oct:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<dev::Octet<__nv_bfloat16>, true>, 128, 0);
        break;
    case kStoreF16Oct:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<dev::Octet<__half>, true>, 128, 0);
        break;
    default: break;
    }
    return e == cudaSuccess ? n : 0;
}

}  // namespace vr

// ===========================================================================
// Host side: batch tables, CUDA graph, autotuner
// ===========================================================================
using namespace vr;
using namespace vr::host;

struct vr_batch_s {
    vr_ctx ctx = nullptr;
    std::vector<vr_volume> vols;
    std::vector<vr_camera> cams;
    std::vector<float2> vol_tf;
    float *out = nullptr;
    int nb = 0, W = 0, H = 0;
    vr_dtype dtype = VR_F32;
    int kind = kStoreF32;  // storage type and cell layout (StorageKind)
    int pw = 8, bps = 0, slots = 16, mode = 0;
    // device tables
    BatchView *d_views = nullptr;
    BrickLaunch *d_vb = nullptr;
    int *d_order = nullptr;
    long long *d_render_begin = nullptr;
    int *d_unit_march = nullptr, *d_unit_comp = nullptr;
    long long *d_bw_begin = nullptr;
    void **d_vol_data = nullptr;
    float2 *d_vol_tf = nullptr;
    float4 *d_ring = nullptr;
    long long ring_px = 0;
    unsigned long long *d_claim = nullptr;
    int *d_march_done = nullptr, *d_comp_done = nullptr;
    BatchParams bp{};
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool counted = false;  // included in the context's live-object count
    int dbg_wait_limit = 0;  // vr_batch_debug_wait: sleeps per wait (0 = default)
    int dbg_wait_extra = 0;  // vr_batch_debug_wait: added to unit 0's composite target
};

namespace {

void free_tables(vr_batch b)
{
    cudaFree(b->d_views);
    cudaFree(b->d_vb);
    cudaFree(b->d_order);
    cudaFree(b->d_render_begin);
    cudaFree(b->d_unit_march);
    cudaFree(b->d_unit_comp);
    cudaFree(b->d_bw_begin);
    b->d_unit_march = nullptr;
    b->d_unit_comp = nullptr;
    b->d_bw_begin = nullptr;
    b->d_views = nullptr;
    b->d_vb = nullptr;
    b->d_order = nullptr;
    b->d_render_begin = nullptr;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Per-view tables for packet width pw, the work-item prefix, the partial ring,
// and a CUDA graph holding the counter resets plus the one persistent launch.
vr_status build(vr_batch b, int pw, int bps, int mode)
{
    vr_ctx ctx = b->ctx;
    free_tables(b);
    vr_volume vol0 = b->vols[0];
    const int nb = b->nb, nv = static_cast<int>(b->cams.size()), nr = static_cast<int>(b->vols.size()) * nv;
    const int tw = 2 * pw, th = 2 * (32 / pw);
    const double nmax = nmax3(vol0->dims);
    std::vector<BatchView> views(nv);
    std::vector<BrickLaunch> vb(static_cast<size_t>(nv) * nb);
    std::vector<int> order(static_cast<size_t>(nv) * nb);
    long long slot_px = 1;
    const double dt = static_cast<double>(ctx->step) / nmax;
    for (int w = 0; w < nv; ++w) {
        const vr_camera &c = b->cams[w];
        Basis Bs;
        make_basis(c, Bs);
        BatchView &V = views[w];
        std::memset(&V, 0, sizeof(V));
        for (int a = 0; a < 3; ++a) {
            V.eye[a] = static_cast<float>(c.eye[a]);
            V.r[a] = static_cast<float>(Bs.r[a]);
            V.u[a] = static_cast<float>(Bs.u[a]);
            V.f[a] = static_cast<float>(Bs.f[a]);
            V.N[a] = static_cast<float>(vol0->dims[a]);
        }
        V.tanx = static_cast<float>(Bs.tanx);
        V.tany = static_cast<float>(Bs.tany);
        V.ow = static_cast<float>(c.ortho_w);
        V.oh = static_cast<float>(c.ortho_h);
        V.ortho = c.ortho ? 1 : 0;
        V.W = c.width;
        V.H = c.height;
        V.inv_W = static_cast<float>(1.0 / c.width);
        V.inv_H = static_cast<float>(1.0 / c.height);
        V.nmax = static_cast<float>(nmax);
        V.dt = static_cast<float>(dt);
        V.inv_dt = static_cast<float>(1.0 / dt);
        std::vector<int> ord;
        visibility_order(vol0->tree, 0, c, nmax, ord);
        std::copy(ord.begin(), ord.end(), order.begin() + static_cast<size_t>(w) * nb);
        long long px = 0;
        int items = 0;
        for (int k = 0; k < nb; ++k) {
            BrickLaunch &L = vb[static_cast<size_t>(w) * nb + k];
            std::memset(&L, 0, sizeof(L));
            const int *bx = &vol0->boxes[6 * k];
            footprint(c, Bs, bx, nmax, L.rect);
            for (int a = 0; a < 3; ++a) {
                L.lo[a] = bx[a];
                L.hi[a] = bx[3 + a];
                L.own_lo[a] = bx[a] == 0 ? -INFINITY : static_cast<float>(bx[a]);
                L.own_hi[a] = bx[3 + a] == vol0->dims[a] ? INFINITY : static_cast<float>(bx[3 + a]);
            }
            L.sx = bx[3] - bx[0] + 2;
            L.sy = bx[4] - bx[1] + 2;
            L.base = vol0->base[k];
            L.poff = px;
            px += static_cast<long long>(L.rect[2]) * L.rect[3];
            px = (px + 7) & ~7LL;
            L.item_begin = items;
            L.tiles_x = (L.rect[2] + tw - 1) / tw;
            items += L.tiles_x * ((L.rect[3] + th - 1) / th);
        }
        V.march_items = items;
        V.comp_items = ((c.width + kBatchCompW - 1) / kBatchCompW) * ((c.height + kBatchCompH - 1) / kBatchCompH);
        slot_px = std::max(slot_px, px);
    }
    // units: renders (mode 0) or volumes with all their views (mode 1, brick-major)
    const int nvol = static_cast<int>(b->vols.size());
    const int nu = mode == 0 ? nr : nvol;
    std::vector<int> unit_march(nu), unit_comp(nu);
    std::vector<long long> bw(static_cast<size_t>(nb) * nv + 1, 0);
    if (mode == 1) {
        for (int k = 0; k < nb; ++k)
            for (int w = 0; w < nv; ++w) {
                const BrickLaunch &L = vb[static_cast<size_t>(w) * nb + k];
                const long long tiles = static_cast<long long>(L.tiles_x) * ((L.rect[3] + th - 1) / th);
                bw[static_cast<size_t>(k) * nv + w + 1] = bw[static_cast<size_t>(k) * nv + w] + tiles;
            }
    }
    for (int u = 0; u < nu; ++u) {
        if (mode == 0) {
            unit_march[u] = views[u % nv].march_items;
            unit_comp[u] = views[u % nv].comp_items;
        } else {
            unit_march[u] = static_cast<int>(bw.back());
            unit_comp[u] = nv * views[0].comp_items;
        }
    }
    // segments: g = 0..nu, segment g = march items of unit g + composite tiles of unit g-1
    std::vector<long long> begin(nu + 2, 0);
    for (int g = 0; g <= nu; ++g) {
        const long long m = g < nu ? unit_march[g] : 0;
        const long long c = g > 0 ? unit_comp[g - 1] : 0;
        begin[g + 1] = begin[g] + m + c;
    }
    DeviceGuard g(ctx->device);
    VR_CUDA(ctx, vr::host::dev_malloc(&b->d_views, views.size() * sizeof(BatchView)));
    VR_CUDA(ctx, vr::host::dev_malloc(&b->d_vb, vb.size() * sizeof(BrickLaunch)));
    VR_CUDA(ctx, vr::host::dev_malloc(&b->d_order, order.size() * sizeof(int)));
    VR_CUDA(ctx, vr::host::dev_malloc(&b->d_render_begin, begin.size() * sizeof(long long)));
    VR_CUDA(ctx, cudaMemcpy(b->d_views, views.data(), views.size() * sizeof(BatchView), cudaMemcpyHostToDevice));
    VR_CUDA(ctx, cudaMemcpy(b->d_vb, vb.data(), vb.size() * sizeof(BrickLaunch), cudaMemcpyHostToDevice));
    VR_CUDA(ctx, cudaMemcpy(b->d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice));
    VR_CUDA(ctx, cudaMemcpy(b->d_render_begin, begin.data(), begin.size() * sizeof(long long), cudaMemcpyHostToDevice));
    VR_CUDA(ctx, vr::host::dev_malloc(&b->d_unit_march, unit_march.size() * sizeof(int)));
    VR_CUDA(ctx, vr::host::dev_malloc(&b->d_unit_comp, unit_comp.size() * sizeof(int)));
    VR_CUDA(ctx, vr::host::dev_malloc(&b->d_bw_begin, bw.size() * sizeof(long long)));
    VR_CUDA(ctx, cudaMemcpy(b->d_unit_march, unit_march.data(), unit_march.size() * sizeof(int), cudaMemcpyHostToDevice));
    VR_CUDA(ctx, cudaMemcpy(b->d_unit_comp, unit_comp.data(), unit_comp.size() * sizeof(int), cudaMemcpyHostToDevice));
    VR_CUDA(ctx, cudaMemcpy(b->d_bw_begin, bw.data(), bw.size() * sizeof(long long), cudaMemcpyHostToDevice));
    // at least two slots: render r's march items wait for the composite of
    // render r - slots, which must lie in an earlier segment
    const int slots = std::max(1, std::min(mode == 0 ? b->slots : 2, nu));
    const long long unit_px = mode == 0 ? slot_px : slot_px * nv;
    const long long need = unit_px * slots;
    if (need > b->ring_px) {
        cudaFree(b->d_ring);
        b->d_ring = nullptr;
        b->ring_px = 0;
        VR_CUDA(ctx, vr::host::dev_malloc(&b->d_ring, static_cast<size_t>(need) * sizeof(float4)));
        b->ring_px = need;
    }
    int sms = 0;
    VR_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const int maxb = batch_max_blocks_per_sm(b->kind);
    if (maxb < 1) return fail(ctx, VR_ERR_CUDA, "batched kernel cannot be resident");
    bps = std::max(1, std::min(bps > 0 ? bps : maxb, maxb));
    b->pw = pw;
    b->bps = bps;
    b->mode = mode;
    BatchParams &p = b->bp;
    std::memset(&p, 0, sizeof(p));
    p.n_renders = nr;
    p.n_units = nu;
    p.mode = mode;
    p.unit_march = b->d_unit_march;
    p.unit_comp = b->d_unit_comp;
    p.bw_begin = b->d_bw_begin;
    p.view_stride = mode == 0 ? 0 : slot_px;
    p.n_views = nv;
    p.nb = nb;
    p.pw = pw;
    p.total_items = begin[nu + 1];
    p.render_begin = b->d_render_begin;
    p.views = b->d_views;
    p.vb = b->d_vb;
    p.order = b->d_order;
    p.vol_data = b->d_vol_data;
    p.vol_tf = b->d_vol_tf;
    p.tf = ctx->d_tf;
    p.ntf = ctx->ntf;
    p.ert_T = ctx->ert_alpha < 1.0f ? static_cast<float>(1.0 - static_cast<double>(ctx->ert_alpha)) : -1.0f;
    p.opc_ratio = ctx->opc_ref > 0.0f ? static_cast<float>(static_cast<double>(ctx->step) / ctx->opc_ref) : 1.0f;
    p.ring = b->d_ring;
    p.slot_px = unit_px;
    p.slots = slots;
    p.out = reinterpret_cast<float4 *>(b->out);
    p.claim = b->d_claim;
    p.march_done = b->d_march_done;
    p.comp_done = b->d_comp_done;
    p.error = ctx->d_error;
    p.wait_limit = b->dbg_wait_limit > 0 ? b->dbg_wait_limit : 1 << 25;  // default: about 4 s of 128 ns sleeps
    p.wait_extra = b->dbg_wait_extra;
    // graph: reset the counters, then the single persistent launch
    VR_CUDA(ctx, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(b->d_claim, 0, sizeof(unsigned long long), b->cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_march_done, 0, nu * sizeof(int), b->cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_comp_done, 0, nu * sizeof(int), b->cap);
    if (e == cudaSuccess && vr::host::fault_now(VR_FAULT_LAUNCH)) e = cudaErrorLaunchFailure;
    if (e == cudaSuccess) e = launch_batch(p, b->kind, sms * bps, b->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(ctx, e != cudaSuccess ? e : e2, "batch graph capture");
    }
    b->graph = graph;
    VR_CUDA(ctx, cudaGraphInstantiate(&b->exec, graph, 0));
    return VR_OK;
}

}  // namespace

extern "C" {

vr_status vr_batch_create(vr_ctx ctx, int n_volumes, const vr_volume *vols, const float *vmins, const float *vmaxs,
                          int n_views, const vr_camera *cams, float *out_rgba_dev, vr_batch *out)
{
    if (!ctx || !out) return VR_ERR_ARG;
    *out = nullptr;
    if (n_volumes < 1 || n_views < 1 || !vols || !cams || !out_rgba_dev)
        return fail(ctx, VR_ERR_ARG, "bad batch description");
    if (!ctx->has_tf) return fail(ctx, VR_ERR_STATE, "no transfer function set");
    if (static_cast<long long>(n_volumes) * n_views > (1 << 20)) return fail(ctx, VR_ERR_ARG, "too many renders");
    vr_volume v0 = vols[0];
    for (int i = 0; i < n_volumes; ++i) {
        const vr_volume v = vols[i];
        if (!v || v->ctx != ctx) return fail(ctx, VR_ERR_ARG, "volume missing or from another context");
        if (std::memcmp(v->dims, v0->dims, sizeof(v0->dims)) != 0 || v->boxes != v0->boxes || v->dtype != v0->dtype)
            return fail(ctx, VR_ERR_ARG, "batched volumes must share dims, partition and storage type");
        if (!v->held.empty()) return fail(ctx, VR_ERR_ARG, "batched volumes must hold every brick (no shares)");
        if (v->octets != v0->octets) return fail(ctx, VR_ERR_ARG, "batched volumes must share the cell layout");
    }
    for (int w = 0; w < n_views; ++w) {
        const vr_camera &c = cams[w];
        Basis Bs;
        if (c.width != cams[0].width || c.height != cams[0].height || c.width < 1 || c.height < 1 ||
            !make_basis(c, Bs) || (c.ortho ? !(c.ortho_w > 0 && c.ortho_h > 0) : !(c.fovy_deg > 0 && c.fovy_deg < 180)))
            return fail(ctx, VR_ERR_ARG, "batched cameras must be valid and share the image size");
    }
    std::unique_ptr<vr_batch_s> b(new (std::nothrow) vr_batch_s);
    if (!b) return VR_ERR_OOM;
    b->ctx = ctx;
    b->vols.assign(vols, vols + n_volumes);
    b->cams.assign(cams, cams + n_views);
    b->out = out_rgba_dev;
    b->nb = static_cast<int>(v0->boxes.size() / 6);
    b->W = cams[0].width;
    b->H = cams[0].height;
    b->dtype = v0->dtype;
    b->kind = storage_kind(v0->dtype, v0->octets);
    for (int i = 0; i < n_volumes; ++i) {
        const double lo = vmins ? vmins[i] : ctx->vmin, hi = vmaxs ? vmaxs[i] : ctx->vmax;
        if (!(hi > lo)) return fail(ctx, VR_ERR_ARG, "batched volume range must have vmax > vmin");
        const double scale = (ctx->ntf - 1) / (hi - lo);
        b->vol_tf.push_back(make_float2(static_cast<float>(scale), static_cast<float>(-lo * scale)));
    }
    DeviceGuard g(ctx->device);
    std::vector<const void *> data(n_volumes);
    for (int i = 0; i < n_volumes; ++i) data[i] = vols[i]->d_data;
    const int nr = n_volumes * n_views;
    cudaError_t e = vr::host::dev_malloc(&b->d_vol_data, n_volumes * sizeof(void *));
    if (e == cudaSuccess) e = vr::host::dev_malloc(&b->d_vol_tf, n_volumes * sizeof(float2));
    if (e == cudaSuccess) e = vr::host::dev_malloc(&b->d_claim, sizeof(unsigned long long));
    if (e == cudaSuccess) e = vr::host::dev_malloc(&b->d_march_done, nr * sizeof(int));
    if (e == cudaSuccess) e = vr::host::dev_malloc(&b->d_comp_done, nr * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_vol_data, data.data(), n_volumes * sizeof(void *), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_vol_tf, b->vol_tf.data(), n_volumes * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    vr_status st = e == cudaSuccess ? build(b.get(), 8, 0, 0) : cuda_fail(ctx, e, "batch setup");
    if (st != VR_OK) {
        vr_batch raw = b.release();
        vr_batch_release(raw);
        return st;
    }
    ctx->live_objects++;
    b->counted = true;
    *out = b.release();
    return VR_OK;
}

vr_status vr_batch_launch(vr_batch b, void *stream)
{
    vr::host::TraceRange trace_("vr_batch_launch");
    if (!b || !b->exec) return VR_ERR_ARG;
    DeviceGuard g(b->ctx->device);
    VR_CUDA(b->ctx, cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
    return VR_OK;
}

vr_status vr_batch_autotune(vr_batch b, void *stream, const char *cache_path, int *chosen)
{
    if (!b) return VR_ERR_ARG;
    vr_ctx ctx = b->ctx;
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaDeviceProp prop;
    VR_CUDA(ctx, cudaGetDeviceProperties(&prop, ctx->device));
    // cache key: device, volumes, views, bricks, image, dims, storage
    char key[512];
    std::snprintf(key, sizeof(key), "%s|v%zu|w%zu|b%d|%dx%d|%dx%dx%d|t%d", prop.name, b->vols.size(), b->cams.size(),
                  b->nb, b->W, b->H, b->vols[0]->dims[0], b->vols[0]->dims[1], b->vols[0]->dims[2],
                  b->kind);
    int best_pw = 0, best_bps = 0, best_mode = 0;
    if (cache_path) {
        if (FILE *f = std::fopen(cache_path, "r")) {
            char line[1024];
            while (std::fgets(line, sizeof(line), f)) {
                char k[512];
                int pw = 0, bps = 0, mode = 0;
                float ms = 0;
                if (std::sscanf(line, "%511s %d %d %d %f", k, &pw, &bps, &mode, &ms) == 5 && std::strcmp(k, key) == 0) {
                    best_pw = pw;
                    best_bps = bps;
                    best_mode = mode;
                }
            }
            std::fclose(f);
        }
    }
    float best_ms = 0.0f;
    if (!best_pw) {
        const int maxb = batch_max_blocks_per_sm(b->kind);
        const int pws[3] = {4, 8, 16};
        std::vector<int> bpss;
        for (int c : {maxb / 2, (3 * maxb) / 4, maxb})
            if (c >= 1 && std::find(bpss.begin(), bpss.end(), c) == bpss.end()) bpss.push_back(c);
        cudaEvent_t e0, e1;
        VR_CUDA(ctx, cudaEventCreate(&e0));
        VR_CUDA(ctx, cudaEventCreate(&e1));
        for (int mode : {0, 1})
        for (int pw : pws)
            for (int bps : bpss) {
                vr_status st = build(b, pw, bps, mode);
                if (st != VR_OK) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return st;
                }
                VR_CUDA(ctx, cudaGraphLaunch(b->exec, s));  // warm
                VR_CUDA(ctx, cudaEventRecord(e0, s));
                VR_CUDA(ctx, cudaGraphLaunch(b->exec, s));
                VR_CUDA(ctx, cudaEventRecord(e1, s));
                VR_CUDA(ctx, cudaEventSynchronize(e1));
                float ms = 0.0f;
                VR_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
                if (!best_pw || ms < best_ms) {
                    best_ms = ms;
                    best_pw = pw;
                    best_bps = b->bps;
                    best_mode = mode;
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (cache_path) {
            if (FILE *f = std::fopen(cache_path, "a")) {
                std::fprintf(f, "%s %d %d %d %.4f\n", key, best_pw, best_bps, best_mode, best_ms);
                std::fclose(f);
            }
        }
    }
    vr_status st = build(b, best_pw, best_bps, best_mode);
    if (st != VR_OK) return st;
    if (chosen) {
        chosen[0] = b->pw;
        chosen[1] = b->bps;
        chosen[2] = b->bp.slots;
        chosen[3] = b->mode;
    }
    return VR_OK;
}

vr_status vr_batch_configure(vr_batch b, int packet_width, int blocks_per_sm, int order)
{
    if (!b) return VR_ERR_ARG;
    if ((packet_width != 4 && packet_width != 8 && packet_width != 16) || blocks_per_sm < 0 ||
        (order != 0 && order != 1))
        return fail(b->ctx, VR_ERR_ARG, "bad batch configuration");
    return build(b, packet_width, blocks_per_sm, order);
}

vr_status vr_batch_debug_wait(vr_batch b, int wait_limit, int extra_march)
{
    if (!b) return VR_ERR_ARG;
    if (wait_limit < 0 || extra_march < 0) return fail(b->ctx, VR_ERR_ARG, "negative wait limit or extra count");
    b->dbg_wait_limit = wait_limit;
    b->dbg_wait_extra = extra_march;
    return build(b, b->pw, b->bps, b->mode);
}

vr_status vr_batch_release(vr_batch b)
{
    if (!b) return VR_ERR_ARG;
    DeviceGuard g(b->ctx->device);
    if (b->cap) cudaStreamSynchronize(b->cap);
    free_tables(b);
    cudaFree(b->d_ring);
    cudaFree(b->d_vol_data);
    cudaFree(b->d_vol_tf);
    cudaFree(b->d_claim);
    cudaFree(b->d_march_done);
    cudaFree(b->d_comp_done);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->counted) b->ctx->live_objects--;
    delete b;
    return VR_OK;
}

}  // extern "C"
