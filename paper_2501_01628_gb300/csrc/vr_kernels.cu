// vr_kernels.cu -- CUDA kernels (sm_103a) of the per-brick emission-absorption
// march and the sort-last "over" composite.
//
// Sec. 2.2 of arXiv:2501.01628: data is spatially distributed, each rank
// renders its share. Sec. 3/4: the per-rank images are composited into one
// framebuffer. The optical model is the standard emission-absorption one; the
// exact per-sample definitions are stated in include/vr.h.
#include "vr_device.cuh"

namespace vr {
namespace {

using dev::Quad;
using dev::find_brick;
using dev::over;

// ---------------------------------------------------------------------------
// Pack: global x-fastest float32 volume -> one brick of xy-quads (halo of one
// voxel, edge-clamped), converted to the storage type with round-to-nearest.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void pack_kernel(PackParams p)
{
    using Q = typename Quad<T>::type;
    Q *dst = static_cast<Q *>(p.dst);
    const int qx = p.s[0] - 1, qy = p.s[1] - 1, nbx = p.s[0] / 2, nby = p.s[1] / 2;
    const long long qxy = static_cast<long long>(qx) * qy;
    const long long count = qxy * p.s[2];
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < count;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int lz = static_cast<int>(e / qxy);
        const long long rem = e - lz * qxy;
        const int ly = static_cast<int>(rem / qx);
        const int lx = static_cast<int>(rem - static_cast<long long>(ly) * qx);
        const int gx0 = min(max(p.lo[0] + lx - 1, 0), p.N[0] - 1);
        const int gx1 = min(max(p.lo[0] + lx, 0), p.N[0] - 1);
        const int gy0 = min(max(p.lo[1] + ly - 1, 0), p.N[1] - 1);
        const int gy1 = min(max(p.lo[1] + ly, 0), p.N[1] - 1);
        const int gz = min(max(p.lo[2] + lz - 1, 0), p.N[2] - 1);
        const float *plane = p.src + static_cast<long long>(gz) * p.N[1] * p.N[0];
        const float *r0 = plane + static_cast<long long>(gy0) * p.N[0];
        const float *r1 = plane + static_cast<long long>(gy1) * p.N[0];
        dst[quad_index(lx, ly, lz, nbx, nby)] = Quad<T>::make(r0[gx0], r0[gx1], r1[gx0], r1[gx1]);
    }
}

// ---------------------------------------------------------------------------
// March: one thread per pixel of a brick's footprint; 8x4-pixel warp packets.
// ---------------------------------------------------------------------------
template <typename S, bool COUNT>
__global__ void __launch_bounds__(128) march_kernel(const __grid_constant__ MarchParams p)
{
    // transfer function as (T[i], T[i+1]-T[i]) pairs; the last difference is 0
    // transfer-function pairs (8 KB for 256 entries) are read through L1: one
    // cached copy per SM instead of one shared-memory copy per block

    const int item = blockIdx.x;
    const int bi = find_brick(p, item);
    const BrickLaunch &B = p.b[bi];
    const int local = item - B.item_begin;
    const int ty = local / B.tiles_x, tx = local - ty * B.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rx = tx * kTileW + (warp & 1) * 8 + (lane & 7);
    const int ry = ty * kTileH + (warp >> 1) * 4 + (lane >> 3);
    if (rx >= B.rect[2] || ry >= B.rect[3]) return;
    const int px = B.rect[0] + rx, py = B.rect[1] + ry;

    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
    unsigned long long executed = 0;
    dev::OwnedRun run;
    dev::owned_run(p, B, px, py, run);
    {
        const int ka = run.ka, kb = run.kb;
        // owned samples are contiguous along the ray: [ka, kb] are all owned
        if (ka <= kb) {
            using Q = typename Quad<S>::type;
            const Q *vox = static_cast<const Q *>(p.data) + B.base;
            const int nbx = B.sx / 2, nby = B.sy / 2;
            const int imax = B.hi[0] - B.lo[0], jmax = B.hi[1] - B.lo[1], kmax = B.hi[2] - B.lo[2];
            const float xmax = static_cast<float>(p.ntf - 1);
            const float *base = run.base, *step = run.step;
            // two samples per iteration: both cells' loads are issued before either
            // sample is classified (independent memory requests in flight)
            int prev = -1;
            float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
            float kh = static_cast<float>(ka) + 0.5f;
            // quad indices of planes k and k+1 of the sample's cell; the clamps
            // only guard memory (owned samples always lie inside the brick)
            auto locate = [&](float h, int &cell, int &cell1, float &wx, float &wy, float &wz) {
                const float vx = fmaf(h, step[0], base[0]);
                const float vy = fmaf(h, step[1], base[1]);
                const float vz = fmaf(h, step[2], base[2]);
                const float flx = floorf(vx), fly = floorf(vy), flz = floorf(vz);
                wx = vx - flx;
                wy = vy - fly;
                wz = vz - flz;
                const int i = min(max(static_cast<int>(flx), 0), imax);
                const int j = min(max(static_cast<int>(fly), 0), jmax);
                const int k = min(max(static_cast<int>(flz), 0), kmax);
                cell = quad_index(i, j, k, nbx, nby);
                cell1 = quad_index(i, j, k + 1, nbx, nby);
            };
            auto shade = [&](const float4 &a0, const float4 &a1, float wx, float wy, float wz) {
                const float c00 = fmaf(wx, a0.y - a0.x, a0.x), c10 = fmaf(wx, a0.w - a0.z, a0.z);
                const float c01 = fmaf(wx, a1.y - a1.x, a1.x), c11 = fmaf(wx, a1.w - a1.z, a1.z);
                const float c0 = fmaf(wy, c10 - c00, c00), c1 = fmaf(wy, c11 - c01, c01);
                const float s = fmaf(wz, c1 - c0, c0);
                const float x = fminf(fmaxf(fmaf(s, p.tf_scale, p.tf_bias), 0.0f), xmax);
                const int ti = static_cast<int>(x);
                const float w = x - static_cast<float>(ti);
                const float4 e0 = __ldg(p.tf + 2 * ti), de = __ldg(p.tf + 2 * ti + 1);
                const float r = fmaf(w, de.x, e0.x), g = fmaf(w, de.y, e0.y);
                const float bb = fmaf(w, de.z, e0.z), al = fmaf(w, de.w, e0.w);
                const float ta = T * al;
                C0 = fmaf(ta, r, C0);
                C1 = fmaf(ta, g, C1);
                C2 = fmaf(ta, bb, C2);
                T = T - ta;
            };
            for (int k = ka; k <= kb; k += 2, kh += 2.0f) {
                int ca, ca1, cb, cb1;
                float ax, ay, az, bx, by, bz;
                locate(kh, ca, ca1, ax, ay, az);
                const bool two = k < kb;
                locate(kh + 1.0f, cb, cb1, bx, by, bz);
                if (ca != prev) {
                    q0 = Quad<S>::load(vox + ca);
                    q1 = Quad<S>::load(vox + ca1);
                }
                float4 r0 = q0, r1 = q1;
                if (two && cb != ca) {
                    r0 = Quad<S>::load(vox + cb);
                    r1 = Quad<S>::load(vox + cb1);
                }
                shade(q0, q1, ax, ay, az);
                if (COUNT) ++executed;
                if (T <= p.ert_T || !two) break;
                shade(r0, r1, bx, by, bz);
                if (COUNT) ++executed;
                if (T <= p.ert_T) break;
                q0 = r0;
                q1 = r1;
                prev = cb;
            }
        }
    }
    p.partials[B.poff + static_cast<long long>(ry) * B.rect[2] + rx] = make_float4(C0, C1, C2, 1.0f - T);
    if (COUNT && executed) atomicAdd(p.sample_counter, executed);
}

// ---------------------------------------------------------------------------
// Composite: one block per 32x8 image tile, one thread per pixel; partials are
// combined front to back with "over" along the configured association tree.
// ---------------------------------------------------------------------------
// Per tile, warp 0 first compacts the bricks whose rectangles overlap the tile,
// in visibility order. Absent partials are the identity of "over", so only the
// association tree's carries at skipped positions matter; consecutive carries
// compose to the deepest one, so each listed brick carries max(carry) up to the
// next listed position.
template <int LEVELS>
__global__ void __launch_bounds__(256) composite_kernel(const __grid_constant__ CompositeParams p)
{
    __shared__ int s_brick[kMaxBricks];
    __shared__ int s_pos[kMaxBricks + 1];
    __shared__ unsigned char s_carry[kMaxBricks];
    __shared__ int s_m;
    const int tx0 = blockIdx.x * kCompW, ty0 = blockIdx.y * kCompH;
    const int tid = threadIdx.y * kCompW + threadIdx.x;
    if (tid < 32) {
        int m = 0;
        for (int j0 = 0; j0 < p.nb; j0 += 32) {
            const int j = j0 + tid;
            bool ov = false;
            int b = 0;
            if (j < p.nb) {
                b = p.order[j];
                const int x0 = p.rect[b][0], y0 = p.rect[b][1], w = p.rect[b][2], h = p.rect[b][3];
                ov = x0 < tx0 + kCompW && tx0 < x0 + w && y0 < ty0 + kCompH && ty0 < y0 + h;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ov);
            if (ov) {
                const int at = m + __popc(bal & ((1u << tid) - 1u));
                s_brick[at] = b;
                s_pos[at] = j;
            }
            m += __popc(bal);
        }
        __syncwarp();
        if (tid == 0) {
            s_m = m;
            s_pos[m] = p.nb;
        }
        __syncwarp();
        if (LEVELS > 1)
            for (int i = tid; i < m; i += 32) {
                int c = 0;
                for (int j = s_pos[i]; j < s_pos[i + 1]; ++j) c = max(c, static_cast<int>(p.carry[j]));
                s_carry[i] = static_cast<unsigned char>(c);
            }
    }
    __syncthreads();
    const int m = s_m;
    const int px = tx0 + threadIdx.x, py = ty0 + threadIdx.y;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 acc[LEVELS];
#pragma unroll
    for (int l = 0; l < LEVELS; ++l) acc[l] = zero;
    constexpr int kBatch = 4;  // partial loads in flight before they are combined
    for (int i0 = 0; i0 < m; i0 += kBatch) {
        float4 v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            v[u] = zero;
            if (i0 + u < m) {
                const int b = s_brick[i0 + u];
                const int x0 = p.rect[b][0], y0 = p.rect[b][1], w = p.rect[b][2], h = p.rect[b][3];
                if (px >= x0 && px < x0 + w && py >= y0 && py < y0 + h)
                    v[u] = __ldcs(p.partials + p.poff[b] + static_cast<long long>(py - y0) * w + (px - x0));
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (i0 + u < m) {
                acc[0] = over(acc[0], v[u]);
                if (LEVELS > 1) {
                    const int c = s_carry[i0 + u];
#pragma unroll
                    for (int l = 0; l + 1 < LEVELS; ++l) {
                        if (l < c) {
                            acc[l + 1] = over(acc[l + 1], acc[l]);
                            acc[l] = zero;
                        }
                    }
                }
            }
        }
    }
    if (px < p.W && py < p.H) {
        float4 r = acc[0];
#pragma unroll
        for (int l = 1; l < LEVELS; ++l)
            if (l == p.n_levels - 1) r = acc[l];
        __stcs(p.out + static_cast<long long>(py) * p.W + px, r);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_pack(const PackParams &p, vr_dtype dtype, cudaStream_t s)
{
    const long long count = static_cast<long long>(p.s[0] - 1) * (p.s[1] - 1) * p.s[2];
    if (count <= 0) return cudaSuccess;
    const int threads = 256;
    long long blocks = (count + threads - 1) / threads;
    if (blocks > 152 * 64) blocks = 152 * 64;
    switch (dtype) {
    case VR_F32: pack_kernel<float><<<static_cast<int>(blocks), threads, 0, s>>>(p); break;
    case VR_BF16: pack_kernel<__nv_bfloat16><<<static_cast<int>(blocks), threads, 0, s>>>(p); break;
    case VR_F16: pack_kernel<__half><<<static_cast<int>(blocks), threads, 0, s>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_march(const MarchParams &p, vr_dtype dtype, cudaStream_t s)
{
    if (p.n_items <= 0) return cudaSuccess;
    const bool count = p.sample_counter != nullptr;
#define VR_MARCH(T)                                                                      \
    (count ? (march_kernel<T, true><<<p.n_items, 128, 0, s>>>(p), 0)                     \
           : (march_kernel<T, false><<<p.n_items, 128, 0, s>>>(p), 0))
    switch (dtype) {
    case VR_F32: VR_MARCH(float); break;
    case VR_BF16: VR_MARCH(__nv_bfloat16); break;
    case VR_F16: VR_MARCH(__half); break;
    default: return cudaErrorInvalidValue;
    }
#undef VR_MARCH
    return cudaGetLastError();
}

cudaError_t launch_composite(const CompositeParams &p, cudaStream_t s)
{
    dim3 block(kCompW, kCompH);
    dim3 grid((p.W + kCompW - 1) / kCompW, (p.H + kCompH - 1) / kCompH);
    if (p.W <= 0 || p.H <= 0) return cudaSuccess;
    if (p.n_levels <= 1) composite_kernel<1><<<grid, block, 0, s>>>(p);
    else if (p.n_levels <= 4) composite_kernel<4><<<grid, block, 0, s>>>(p);
    else composite_kernel<kMaxFactors><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace vr
