// vr_composite.cu -- CUDA kernels (sm_103a) of the sort-last "over" composite:
// the per-brick partial images combined front to back into one framebuffer
// (Sec. 3/4 of arXiv:2501.01628), and the composite of whole rank images used
// by the exchange rounds between GPUs.
#include <algorithm>

#include "vr_device.cuh"

namespace vr {
namespace {

using dev::over;

// Stand-alone mask pass, for frames whose march does not write the masks.
__global__ void __launch_bounds__(kMaskThreads) tile_mask_kernel(const __grid_constant__ CompositeParams p)
{
    dev::write_tile_mask(blockIdx.x * kMaskThreads + threadIdx.x, p.tiles_x, p.tiles_y, p.nb, p.order,
                    [&](int b) { return make_int4(p.rect[b][0], p.rect[b][1], p.rect[b][2], p.rect[b][3]); },
                    p.tile_mask);
}

// ---------------------------------------------------------------------------
// Composite: one 32x8-thread block per kCompW x kCompTileH (32 x 8) image tile,
// or a persistent grid whose blocks take tiles in turn; one thread per pixel.
// Partials are combined front to back with "over" along the configured
// association tree.
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
    {
        const int py = ty0 + threadIdx.y;
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
    if (p.pool_done) {
        // pipelined frames: once every block has read its partials, the last
        // block to finish releases the pool to the frame after next
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            __threadfence();
            if (atomicAdd(p.pool_count + p.pool, 1u) == gridDim.x - 1) {
                p.pool_count[p.pool] = 0;  // for the pool's next composite
                asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p.pool_done + p.pool), "l"(p.pool_frame)
                             : "memory");
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
