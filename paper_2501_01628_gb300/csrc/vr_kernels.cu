// vr_kernels.cu -- CUDA kernels (sm_103a) of the brick pack and the per-brick
// emission-absorption march (the sort-last "over" composite is in
// vr_composite.cu, the ray-state cycling frame in vr_cycle.cu).
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
    // it waits; its writes (masks, partials) go to a pool that the frame before
    // the previous one read. The mask blocks wait for the preceding grid's
    // completion (so this grid completes only after it); the march blocks wait
    // only for the composite that last read their pool (pool_ready). Outside
    // such a launch both waits return at once.
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
    if (!dev::pool_ready(p.pool_done, p.pool, p.pool_frame, p.count_error)) return;
    unsigned long long policy;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(policy));
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(dst), "f"(c.x), "f"(c.y),
                 "f"(c.z), "f"(c.w), "l"(policy)
                 : "memory");
    if (COUNT && executed) atomicAdd(p.sample_counter, executed);
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

}  // namespace vr
