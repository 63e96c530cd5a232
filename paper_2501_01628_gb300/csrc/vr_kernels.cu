// vr_kernels.cu -- CUDA kernels (sm_103a) of the per-brick emission-absorption
// march and the sort-last "over" composite.
//
// Sec. 2.2 of arXiv:2501.01628: data is spatially distributed, each rank
// renders its share. Sec. 3/4: the per-rank images are composited into one
// framebuffer. The optical model is the standard emission-absorption one; the
// exact per-sample definitions are stated in include/vr.h.
#include <algorithm>

#include "vr_device.cuh"

namespace vr {
namespace {

using dev::Quad;
using dev::find_brick;
using dev::over;

// ---------------------------------------------------------------------------
// Pack: global x-fastest float32 volume -> every brick's xy-quads (halo of one
// voxel, edge-clamped), converted to the storage type with round-to-nearest.
// One launch for all bricks; a block writes kPackChunk consecutive quads of one
// brick's storage (2x2x2 blocks of quads, blocks x-fastest), so a warp's writes
// are contiguous. Quads of the padding that rounds a brick's storage up to
// whole blocks are not written.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) pack_kernel(const __grid_constant__ PackParams p)
{
    int lo = 0, hi = p.nb - 1;  // the block's brick (the same for all its threads)
    const int blk = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.b[mid].block_begin <= blk) lo = mid;
        else hi = mid - 1;
    }
    const PackBrick &B = p.b[lo];
    using Q = typename Quad<T>::type;
    Q *dst = static_cast<Q *>(B.dst);
    const int qx = B.s[0] - 1, qy = B.s[1] - 1, nbx = B.s[0] / 2, nby = B.s[1] / 2;
    const long long q0 = static_cast<long long>(blk - B.block_begin) * kPackChunk;
    const long long q1 = min(q0 + kPackChunk, B.quads);
    for (long long q = q0 + threadIdx.x; q < q1; q += 256) {
        // inverse of quad_index
        const long long bl = q >> 3;
        const int bx = static_cast<int>(bl % nbx);
        const long long rest = bl / nbx;
        const int by = static_cast<int>(rest % nby);
        const int bz = static_cast<int>(rest / nby);
        const int lx = 2 * bx + static_cast<int>(q & 1), ly = 2 * by + static_cast<int>((q >> 1) & 1);
        const int lz = 2 * bz + static_cast<int>((q >> 2) & 1);
        if (lx >= qx || ly >= qy || lz >= B.s[2]) continue;
        const int gx0 = min(max(B.lo[0] + lx - 1, 0), p.N[0] - 1);
        const int gx1 = min(max(B.lo[0] + lx, 0), p.N[0] - 1);
        const int gy0 = min(max(B.lo[1] + ly - 1, 0), p.N[1] - 1);
        const int gy1 = min(max(B.lo[1] + ly, 0), p.N[1] - 1);
        const int gz = min(max(B.lo[2] + lz - 1, 0), p.N[2] - 1);
        const float *plane = p.src + static_cast<long long>(gz) * p.N[1] * p.N[0];
        const float *r0 = plane + static_cast<long long>(gy0) * p.N[0];
        const float *r1 = plane + static_cast<long long>(gy1) * p.N[0];
        if constexpr (Quad<T>::octet) {  // plane lz and plane lz + 1 in one element
            const int gz1 = min(max(B.lo[2] + lz, 0), p.N[2] - 1);
            const float *plane1 = p.src + static_cast<long long>(gz1) * p.N[1] * p.N[0];
            const float *s0 = plane1 + static_cast<long long>(gy0) * p.N[0];
            const float *s1 = plane1 + static_cast<long long>(gy1) * p.N[0];
            dst[q] = Quad<T>::make8(__ldg(r0 + gx0), __ldg(r0 + gx1), __ldg(r1 + gx0), __ldg(r1 + gx1),
                                    __ldg(s0 + gx0), __ldg(s0 + gx1), __ldg(s1 + gx0), __ldg(s1 + gx1));
        } else {
            dst[q] = Quad<T>::make(__ldg(r0 + gx0), __ldg(r0 + gx1), __ldg(r1 + gx0), __ldg(r1 + gx1));
        }
    }
}

// Stand-alone mask pass, for frames whose march does not write the masks.
__global__ void __launch_bounds__(kMaskThreads) tile_mask_kernel(const __grid_constant__ CompositeParams p)
{
    dev::write_tile_mask(blockIdx.x * kMaskThreads + threadIdx.x, p.tiles_x, p.tiles_y, p.nb, p.order,
                    [&](int b) { return make_int4(p.rect[b][0], p.rect[b][1], p.rect[b][2], p.rect[b][3]); },
                    p.tile_mask);
}

// ---------------------------------------------------------------------------
// March: one thread per pixel of a brick's footprint. A block is a tile of
// 2x2 warp packets of pw x (32/pw) pixels (pw = p.pw: 4, 8 or 16). The transfer
// function is read as (T[i], T[i+1]-T[i]) pairs (the last difference is 0)
// through L1: one cached copy per SM instead of one shared-memory copy per block.
// ---------------------------------------------------------------------------
template <typename S, bool COUNT, bool OPC>
__global__ void __launch_bounds__(128) march_kernel(const __grid_constant__ MarchParams p)
{
    // the composite launched after this march may start once every block of
    // this grid is running; it reads the masks and partials only after this
    // grid has completed
    asm volatile("griddepcontrol.launch_dependents;");
    // Launched as a programmatic dependent of the previous frame's composite
    // (pipelined frames), this grid reads only the bricks and the table before
    // the waits below; its writes (masks, partials) go to a pool that the frame
    // before the previous one read, and wait for the preceding grid's completion.
    // Outside such a launch the waits return at once.
    if (static_cast<int>(blockIdx.x) < p.mask_blocks) {  // the composite's tile masks
        asm volatile("griddepcontrol.wait;" ::: "memory");
        dev::write_tile_mask(blockIdx.x * kMaskThreads + threadIdx.x, p.mask_tiles_x, p.mask_tiles_y, p.nb, p.order,
                        [&](int b) { return make_int4(p.b[b].rect[0], p.b[b].rect[1], p.b[b].rect[2],
                                                      p.b[b].rect[3]); },
                        p.tile_mask);
        return;
    }
    const int item = blockIdx.x - p.mask_blocks;
    const int bi = find_brick(p, item);
    const BrickLaunch &B = p.b[bi];
    const int local = item - B.item_begin;
    const int ty = local / B.tiles_x, tx = local - ty * B.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rx = tx * p.tile_w + (warp & 1) * p.pw + (lane & (p.pw - 1));
    const int ry = ty * p.tile_h + (warp >> 1) * (32 / p.pw) + lane / p.pw;
    if (rx >= B.rect[2] || ry >= B.rect[3]) return;
    const int px = B.rect[0] + rx, py = B.rect[1] + ry;

    unsigned long long executed = 0;
    dev::OwnedRun run;
    dev::owned_run(p, B, px, py, run);
    const float4 c =
        dev::march_run<S, COUNT, OPC>(p.data, B, run, p.tf, p.tf_scale, p.tf_bias, p.ntf, p.ert_T, executed, p.opc_ratio,
                                      p.count_error);
    // the composite reads the partial next: keep it in L2 ahead of the streamed bricks
    float4 *dst = p.partials + B.poff + static_cast<long long>(ry) * B.rect[2] + rx;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    unsigned long long policy;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(policy));
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(dst), "f"(c.x), "f"(c.y),
                 "f"(c.z), "f"(c.w), "l"(policy)
                 : "memory");
    if (COUNT && executed) atomicAdd(p.sample_counter, executed);
}

// ---------------------------------------------------------------------------
// Ray-state cycling: one thread per image pixel carries (C, T) through the
// bricks in front-to-back order (the paper's ray-queue cycling, Sec. 2.2 and 3,
// where every ray visits every rank, restated for bricks on one GPU). No
// partial images and no composite; early termination is global.
// ---------------------------------------------------------------------------
template <typename S, bool COUNT, bool OPC>
__global__ void __launch_bounds__(128) march_cycle_kernel(const __grid_constant__ MarchParams p, float4 *out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px = blockIdx.x * p.tile_w + (warp & 1) * p.pw + (lane & (p.pw - 1));
    const int py = blockIdx.y * p.tile_h + (warp >> 1) * (32 / p.pw) + lane / p.pw;
    if (px >= p.W || py >= p.H) return;
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
    unsigned long long executed = 0;
    dev::Ray ray;
    dev::ray_setup(p, px, py, ray);  // once per pixel; each brick only intersects it
    for (int j = 0; ray.hit && j < p.nb; ++j) {
        const BrickLaunch &B = p.b[p.order[j]];
        if (px < B.rect[0] || px >= B.rect[0] + B.rect[2] || py < B.rect[1] || py >= B.rect[1] + B.rect[3])
            continue;
        dev::OwnedRun run;
        dev::brick_run(p, B, ray, run);
        dev::march_accumulate<S, COUNT, OPC>(p.data, B, run, p.tf, p.tf_scale, p.tf_bias, p.ntf, p.ert_T, C0, C1,
                                             C2, T, executed, p.opc_ratio, p.count_error);
        if (T <= p.ert_T) break;
    }
    out[static_cast<long long>(py) * p.W + px] = make_float4(C0, C1, C2, 1.0f - T);
    if (COUNT && executed) atomicAdd(p.sample_counter, executed);
}

// ---------------------------------------------------------------------------
// Composite: one 32x8-thread block per kCompW x kCompTileH image tile; the
// tile's kCompRows 32x8 slabs in turn, one thread per pixel. Partials are
// combined front to back with "over" along the configured association tree.
// ---------------------------------------------------------------------------
// The tile's mask (one 16-byte load, the same for the whole block) lists the
// visibility positions of the bricks that overlap it, so no block compacts a
// brick list of its own. Partial loads of four listed bricks are in flight
// together. Absent partials are the identity of "over", so only the tree's
// carries at skipped positions matter, and consecutive carries compose to the
// deepest one: before the brick at position j, after the previous listed
// position i, every level whose group changes between i and j is merged.

// The deepest level of the association tree whose group changes between
// visibility positions i < j: gid[q] holds q's group index at level l (groups
// of factors[0] x ... x factors[l-1] positions) in byte l - 1, so it is the
// highest byte in which gid[i] and gid[j] differ (0: none -- same level-1 group).
__device__ __forceinline__ int carried_levels(const CompositeParams &p, int i, int j)
{
    const unsigned long long x = p.gid[i] ^ p.gid[j];
    return x ? (71 - __clzll(static_cast<long long>(x))) >> 3 : 0;
}

// next listed position (-1 when none is left)
__device__ __forceinline__ int next_pos(unsigned long long &r0, unsigned long long &r1)
{
    int q = -1;
    if (r0) {
        q = __ffsll(static_cast<long long>(r0)) - 1;
        r0 &= r0 - 1;
    } else if (r1) {
        q = 63 + __ffsll(static_cast<long long>(r1));
        r1 &= r1 - 1;
    }
    return q;
}

template <int LEVELS>
__global__ void __launch_bounds__(256) composite_kernel(const __grid_constant__ CompositeParams p)
{
    constexpr int kBatch = 4;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    // a march launched after this grid as its programmatic dependent (the next
    // pipelined frame) may start once every block of this grid is running
    asm volatile("griddepcontrol.launch_dependents;");
    // launched as a programmatic dependent of the march: wait for the preceding
    // grid's completion and memory (the masks and partials are its output)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int ntiles = p.tiles_x * p.tiles_y;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {  // one tile per block, or a persistent grid
    const int tyi = tile / p.tiles_x;
    const int tx0 = (tile - tyi * p.tiles_x) * kCompW, ty0 = tyi * kCompTileH;
    const int px = tx0 + threadIdx.x;
    const uint4 mk = __ldg(p.tile_mask + tile);
    for (int half = 0; half < kCompRows; ++half) {
        const int py = ty0 + threadIdx.y + kCompH * half;
        unsigned long long r0 = static_cast<unsigned long long>(mk.x) | (static_cast<unsigned long long>(mk.y) << 32);
        unsigned long long r1 = static_cast<unsigned long long>(mk.z) | (static_cast<unsigned long long>(mk.w) << 32);
        float4 acc[LEVELS];
#pragma unroll
        for (int l = 0; l < LEVELS; ++l) acc[l] = zero;
        int prev = -1;
        while (r0 | r1) {
            int pos[kBatch];
            float4 v[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                pos[u] = next_pos(r0, r1);
                v[u] = zero;
                if (pos[u] >= 0) {
                    const int b = p.order[pos[u]];
                    const int x0 = p.rect[b][0], y0 = p.rect[b][1], w = p.rect[b][2], h = p.rect[b][3];
                    if (px >= x0 && px < x0 + w && py >= y0 && py < y0 + h)
                        v[u] = __ldcs(p.partials + p.poff[b] + static_cast<long long>(py - y0) * w + (px - x0));
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                if (pos[u] >= 0) {
                    if (LEVELS > 1 && prev >= 0) {
                        const int c = carried_levels(p, prev, pos[u]);
                        if (c > 0) {  // uniform: most listed bricks close no group
#pragma unroll
                            for (int l = 0; l + 1 < LEVELS; ++l)
                                if (l < c) {
                                    acc[l + 1] = over(acc[l + 1], acc[l]);
                                    acc[l] = zero;
                                }
                        }
                    }
                    acc[0] = over(acc[0], v[u]);
                    prev = pos[u];
                }
            }
        }
        if (LEVELS > 1 && prev >= 0) {
            const int c = carried_levels(p, prev, p.nb);
#pragma unroll
            for (int l = 0; l + 1 < LEVELS; ++l)
                if (l < c) {
                    acc[l + 1] = over(acc[l + 1], acc[l]);
                    acc[l] = zero;
                }
        }
        if (px < p.W && py < p.H) {
            // after the last carry every level but n_levels - 1 is exactly zero,
            // and "over" with a zero operand is exact: folding all levels gives
            // that level bit for bit, with static indices (a selected index would
            // put the accumulators in local memory)
            float4 res = acc[LEVELS - 1];
#pragma unroll
            for (int l = LEVELS - 2; l >= 0; --l) res = over(res, acc[l]);
            __stcs(p.out + static_cast<long long>(py) * p.W + px, res);
        }
    }
    }
}

// ---------------------------------------------------------------------------
// Images of ranks (shares of the bricks) composited front to back: the step of
// each radix-k exchange round between GPUs (Sec. 3: the ranks' images end up
// composited in one framebuffer). Grid-stride over pixels; every input pixel is
// read once, so a pixel's output may overwrite its first input.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) composite_images_kernel(const __grid_constant__ ImagesParams p)
{
    const long long stride = static_cast<long long>(gridDim.x) * 256;
    for (long long i = static_cast<long long>(blockIdx.x) * 256 + threadIdx.x; i < p.pixels; i += stride) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = 0; j < p.n; ++j) acc = over(acc, __ldcs(p.img[j] + i));
        __stcs(p.out + i, acc);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_pack(const PackParams &p, int kind, cudaStream_t s)
{
    if (p.n_blocks <= 0) return cudaSuccess;
    switch (kind) {
    case kStoreF32: pack_kernel<float><<<p.n_blocks, 256, 0, s>>>(p); break;
    case kStoreBF16: pack_kernel<__nv_bfloat16><<<p.n_blocks, 256, 0, s>>>(p); break;
    case kStoreF16: pack_kernel<__half><<<p.n_blocks, 256, 0, s>>>(p); break;
    case kStoreBF16Oct: pack_kernel<dev::Octet<__nv_bfloat16>><<<p.n_blocks, 256, 0, s>>>(p); break;
    case kStoreF16Oct: pack_kernel<dev::Octet<__half>><<<p.n_blocks, 256, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_march(const MarchParams &p, int kind, cudaStream_t s, bool after_composite)
{
    if (p.n_items + p.mask_blocks <= 0) return cudaSuccess;
    const int grid = p.n_items + p.mask_blocks;
    const bool count = p.sample_counter != nullptr;
    const bool opc = p.opc_ratio != 1.0f;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(128);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = after_composite ? 1 : 0;
#define VR_MARCH(T)                                                                                     \
    (opc ? (count ? cudaLaunchKernelEx(&cfg, march_kernel<T, true, true>, p)                       \
                  : cudaLaunchKernelEx(&cfg, march_kernel<T, false, true>, p))                     \
         : (count ? cudaLaunchKernelEx(&cfg, march_kernel<T, true, false>, p)                      \
                  : cudaLaunchKernelEx(&cfg, march_kernel<T, false, false>, p)))
    cudaError_t e = cudaErrorInvalidValue;
    switch (kind) {
    case kStoreF32: e = VR_MARCH(float); break;
    case kStoreBF16: e = VR_MARCH(__nv_bfloat16); break;
    case kStoreF16: e = VR_MARCH(__half); break;
    case kStoreBF16Oct: e = VR_MARCH(dev::Octet<__nv_bfloat16>); break;
    case kStoreF16Oct: e = VR_MARCH(dev::Octet<__half>); break;
    default: return cudaErrorInvalidValue;
    }
#undef VR_MARCH
    return e;
}

cudaError_t launch_march_cycle(const MarchParams &p, int kind, float4 *out, cudaStream_t s)
{
    if (p.W <= 0 || p.H <= 0) return cudaSuccess;
    const dim3 grid((p.W + p.tile_w - 1) / p.tile_w, (p.H + p.tile_h - 1) / p.tile_h);
    const bool count = p.sample_counter != nullptr;
    const bool opc = p.opc_ratio != 1.0f;
#define VR_CYCLE(T)                                                                                    \
    (opc ? (count ? (march_cycle_kernel<T, true, true><<<grid, 128, 0, s>>>(p, out), 0)                \
                  : (march_cycle_kernel<T, false, true><<<grid, 128, 0, s>>>(p, out), 0))              \
         : (count ? (march_cycle_kernel<T, true, false><<<grid, 128, 0, s>>>(p, out), 0)               \
                  : (march_cycle_kernel<T, false, false><<<grid, 128, 0, s>>>(p, out), 0)))
    switch (kind) {
    case kStoreF32: VR_CYCLE(float); break;
    case kStoreBF16: VR_CYCLE(__nv_bfloat16); break;
    case kStoreF16: VR_CYCLE(__half); break;
    case kStoreBF16Oct: VR_CYCLE(dev::Octet<__nv_bfloat16>); break;
    case kStoreF16Oct: VR_CYCLE(dev::Octet<__half>); break;
    default: return cudaErrorInvalidValue;
    }
#undef VR_CYCLE
    return cudaGetLastError();
}

cudaError_t launch_composite_images(const ImagesParams &p, cudaStream_t s)
{
    if (p.pixels <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long blocks = std::min<long long>((p.pixels + 255) / 256, static_cast<long long>(sms) * 8);
    composite_images_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_tile_masks(const CompositeParams &p, cudaStream_t s)
{
    const int tiles = p.tiles_x * p.tiles_y;
    if (tiles <= 0) return cudaSuccess;
    tile_mask_kernel<<<(tiles + kMaskThreads - 1) / kMaskThreads, kMaskThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_composite(const CompositeParams &p, cudaStream_t s, int max_blocks)
{
    if (p.W <= 0 || p.H <= 0) return cudaSuccess;
    if (p.tiles_x != (p.W + kCompW - 1) / kCompW || p.tiles_y != (p.H + kCompTileH - 1) / kCompTileH ||
        !p.tile_mask)
        return cudaErrorInvalidValue;
    const int tiles = p.tiles_x * p.tiles_y;
    dim3 block(kCompW, kCompH);
    dim3 grid(max_blocks > 0 ? std::min(tiles, max_blocks) : tiles);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    switch (p.n_levels) {  // accumulators for exactly the tree's depth (registers bound the occupancy)
    case 0:
    case 1: return cudaLaunchKernelEx(&cfg, composite_kernel<1>, p);
    case 2: return cudaLaunchKernelEx(&cfg, composite_kernel<2>, p);
    case 3: return cudaLaunchKernelEx(&cfg, composite_kernel<3>, p);
    case 4: return cudaLaunchKernelEx(&cfg, composite_kernel<4>, p);
    default: return cudaLaunchKernelEx(&cfg, composite_kernel<kMaxFactors>, p);
    }
}

}  // namespace vr
