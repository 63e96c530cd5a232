// vr_kernels.cu -- CUDA kernels (sm_103a) of the per-brick emission-absorption
// march and the sort-last "over" composite.
//
// Sec. 2.2 of arXiv:2501.01628: data is spatially distributed, each rank
// renders its share. Sec. 3/4: the per-rank images are composited into one
// framebuffer. The optical model is the standard emission-absorption one; the
// exact per-sample definitions are stated in include/vr.h.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "vr_internal.h"

namespace vr {
namespace {

// ---------------------------------------------------------------------------
// Storage element loads (read-only path)
// ---------------------------------------------------------------------------
template <typename T> struct Elem;
template <> struct Elem<float> {
    static __device__ __forceinline__ float load(const float *p) { return __ldg(p); }
};
template <> struct Elem<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const __nv_bfloat16 *p)
    {
        unsigned short u = __ldg(reinterpret_cast<const unsigned short *>(p));
        return __uint_as_float(static_cast<unsigned>(u) << 16);
    }
};
template <> struct Elem<__half> {
    static __device__ __forceinline__ float load(const __half *p) { return __half2float(__ldg(p)); }
};

// ---------------------------------------------------------------------------
// Pack: global x-fastest float32 volume -> one haloed brick in storage type
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T to_storage(float v);
template <> __device__ __forceinline__ float to_storage<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_storage<__nv_bfloat16>(float v)
{
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half to_storage<__half>(float v) { return __float2half_rn(v); }

template <typename T>
__global__ void pack_kernel(PackParams p)
{
    T *dst = static_cast<T *>(p.dst);
    const long long sxy = static_cast<long long>(p.s[0]) * p.s[1];
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < p.count;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        int lz = static_cast<int>(e / sxy);
        long long rem = e - lz * sxy;
        int ly = static_cast<int>(rem / p.s[0]);
        int lx = static_cast<int>(rem - static_cast<long long>(ly) * p.s[0]);
        int gx = min(max(p.lo[0] + lx - 1, 0), p.N[0] - 1);
        int gy = min(max(p.lo[1] + ly - 1, 0), p.N[1] - 1);
        int gz = min(max(p.lo[2] + lz - 1, 0), p.N[2] - 1);
        float v = p.src[(static_cast<long long>(gz) * p.N[1] + gy) * p.N[0] + gx];
        dst[e] = to_storage<T>(v);
    }
}

// ---------------------------------------------------------------------------
// March: one thread per pixel of a brick's footprint; 8x4-pixel warp packets.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_brick(const MarchParams &p, int item)
{
    int lo = 0, hi = p.nb - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (p.b[mid].item_begin <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename S, bool COUNT>
__global__ void __launch_bounds__(128) march_kernel(const __grid_constant__ MarchParams p)
{
    extern __shared__ float4 s_tf[];
    for (int i = threadIdx.x; i < p.ntf; i += blockDim.x) s_tf[i] = p.tf[i];
    __syncthreads();

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

    // primary ray (FP32; identical arithmetic for every brick)
    const float fx = (static_cast<float>(px) + 0.5f) / static_cast<float>(p.W);
    const float fy = (static_cast<float>(py) + 0.5f) / static_cast<float>(p.H);
    float o[3], d[3];
    if (p.ortho) {
        const float a = (fx - 0.5f) * p.ow, b = (fy - 0.5f) * p.oh;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            o[i] = fmaf(b, p.u[i], fmaf(a, p.r[i], p.eye[i]));
            d[i] = p.f[i];
        }
    } else {
        const float sx = (fx * 2.0f - 1.0f) * p.tanx, sy = (fy * 2.0f - 1.0f) * p.tany;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            o[i] = p.eye[i];
            d[i] = fmaf(sy, p.u[i], fmaf(sx, p.r[i], p.f[i]));
        }
        const float inv = 1.0f / sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
        for (int i = 0; i < 3; ++i) d[i] *= inv;
    }
    // voxel-space origin and direction; t stays in world units
    float ov[3], dv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ov[i] = o[i] * p.nmax;
        dv[i] = d[i] * p.nmax;
    }

    // whole-volume interval [t_in, t_out) and this brick's slab interval
    float t0 = 0.0f, t1 = 3.0e38f, b0 = 0.0f, b1 = 3.0e38f;
    bool hit = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (dv[i] == 0.0f) {
            if (ov[i] < 0.0f || ov[i] > p.N[i]) hit = false;
            if (ov[i] < static_cast<float>(B.lo[i]) || ov[i] > static_cast<float>(B.hi[i])) hit = false;
        } else {
            const float inv = 1.0f / dv[i];
            float ta = (0.0f - ov[i]) * inv, tb = (p.N[i] - ov[i]) * inv;
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
            ta = (static_cast<float>(B.lo[i]) - ov[i]) * inv;
            tb = (static_cast<float>(B.hi[i]) - ov[i]) * inv;
            b0 = fmaxf(b0, fminf(ta, tb));
            b1 = fminf(b1, fmaxf(ta, tb));
        }
    }
    // NOTE: the whole-volume t_in must not depend on the brick; it uses
    // (0 - o)/d and (N - o)/d only, in the same order for every brick.
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
    unsigned long long executed = 0;
    if (hit && t0 < t1 && b0 <= b1) {
        const float t_in = t0, t_out = t1;
        int k_first = max(0, static_cast<int>(floorf((b0 - t_in) * p.inv_dt - 0.5f)) - 1);
        int k_last = static_cast<int>(ceilf((fminf(b1, t_out) - t_in) * p.inv_dt - 0.5f)) + 1;
        const S *vox = static_cast<const S *>(p.data) + B.base;
        const int sx = B.sx, sxy = B.sx * B.sy;
        bool entered = false;
        for (int k = k_first; k <= k_last; ++k) {
            const float t = fmaf(static_cast<float>(k) + 0.5f, p.dt, t_in);
            if (!(t < t_out)) break;
            const float qx = fmaf(t, dv[0], ov[0]);
            const float qy = fmaf(t, dv[1], ov[1]);
            const float qz = fmaf(t, dv[2], ov[2]);
            const bool own = qx >= B.own_lo[0] && qx < B.own_hi[0] && qy >= B.own_lo[1] &&
                             qy < B.own_hi[1] && qz >= B.own_lo[2] && qz < B.own_hi[2];
            if (!own) {
                if (entered) break;
                continue;
            }
            entered = true;
            // trilinear, clamp-to-edge through the halo
            const float vx = qx - 0.5f, vy = qy - 0.5f, vz = qz - 0.5f;
            const float flx = floorf(vx), fly = floorf(vy), flz = floorf(vz);
            const float wx = vx - flx, wy = vy - fly, wz = vz - flz;
            const int ix = min(max(static_cast<int>(flx), B.lo[0] - 1), B.hi[0] - 1) - B.lo[0] + 1;
            const int iy = min(max(static_cast<int>(fly), B.lo[1] - 1), B.hi[1] - 1) - B.lo[1] + 1;
            const int iz = min(max(static_cast<int>(flz), B.lo[2] - 1), B.hi[2] - 1) - B.lo[2] + 1;
            const S *q = vox + (iz * sxy + iy * sx + ix);
            const float v000 = Elem<S>::load(q), v100 = Elem<S>::load(q + 1);
            const float v010 = Elem<S>::load(q + sx), v110 = Elem<S>::load(q + sx + 1);
            const float v001 = Elem<S>::load(q + sxy), v101 = Elem<S>::load(q + sxy + 1);
            const float v011 = Elem<S>::load(q + sxy + sx), v111 = Elem<S>::load(q + sxy + sx + 1);
            const float c00 = fmaf(wx, v100 - v000, v000), c10 = fmaf(wx, v110 - v010, v010);
            const float c01 = fmaf(wx, v101 - v001, v001), c11 = fmaf(wx, v111 - v011, v011);
            const float c0 = fmaf(wy, c10 - c00, c00), c1 = fmaf(wy, c11 - c01, c01);
            const float s = fmaf(wz, c1 - c0, c0);
            // classification
            const float uu = fminf(fmaxf((s - p.vmin) * p.inv_range, 0.0f), 1.0f);
            const float x = uu * static_cast<float>(p.ntf - 1);
            const int ti = min(static_cast<int>(x), p.ntf - 2);
            const float w = x - static_cast<float>(ti);
            const float4 e0 = s_tf[ti], e1 = s_tf[ti + 1];
            const float r = fmaf(w, e1.x - e0.x, e0.x), g = fmaf(w, e1.y - e0.y, e0.y);
            const float bb = fmaf(w, e1.z - e0.z, e0.z), al = fmaf(w, e1.w - e0.w, e0.w);
            // front-to-back emission-absorption
            const float ta = T * al;
            C0 = fmaf(ta, r, C0);
            C1 = fmaf(ta, g, C1);
            C2 = fmaf(ta, bb, C2);
            T = T - ta;
            if (COUNT) ++executed;
            if (T <= p.ert_T) break;
        }
    }
    p.partials[B.poff + static_cast<long long>(ry) * B.rect[2] + rx] = make_float4(C0, C1, C2, 1.0f - T);
    if (COUNT && executed) atomicAdd(p.sample_counter, executed);
}

// ---------------------------------------------------------------------------
// Composite: one block per 32x8 image tile, one thread per pixel; partials are
// combined front to back with "over" along the configured association tree.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 over(float4 front, float4 back)
{
    const float w = 1.0f - front.w;
    return make_float4(fmaf(w, back.x, front.x), fmaf(w, back.y, front.y), fmaf(w, back.z, front.z),
                       fmaf(w, back.w, front.w));
}

template <int LEVELS>
__global__ void __launch_bounds__(256) composite_kernel(const __grid_constant__ CompositeParams p)
{
    const int px = blockIdx.x * kCompW + threadIdx.x;
    const int py = blockIdx.y * kCompH + threadIdx.y;
    const int tx0 = blockIdx.x * kCompW, ty0 = blockIdx.y * kCompH;
    float4 acc[LEVELS];
#pragma unroll
    for (int l = 0; l < LEVELS; ++l) acc[l] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j = 0; j < p.nb; ++j) {
        const int b = p.order[j];
        const int x0 = p.rect[b][0], y0 = p.rect[b][1], w = p.rect[b][2], h = p.rect[b][3];
        // block-uniform overlap test, then per-pixel containment
        if (x0 < tx0 + kCompW && tx0 < x0 + w && y0 < ty0 + kCompH && ty0 < y0 + h) {
            if (px >= x0 && px < x0 + w && py >= y0 && py < y0 + h && px < p.W && py < p.H) {
                const float4 v = p.partials[p.poff[b] + static_cast<long long>(py - y0) * w + (px - x0)];
                acc[0] = over(acc[0], v);
            }
        }
        if (LEVELS > 1) {
            const int c = p.carry[j];
#pragma unroll
            for (int l = 0; l + 1 < LEVELS; ++l) {
                if (l < c) {
                    acc[l + 1] = over(acc[l + 1], acc[l]);
                    acc[l] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
    }
    if (px < p.W && py < p.H) {
        float4 r = acc[0];
        if (LEVELS > 1) {
#pragma unroll
            for (int l = 1; l < LEVELS; ++l)
                if (l == p.n_levels - 1) r = acc[l];
        }
        p.out[static_cast<long long>(py) * p.W + px] = r;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
cudaError_t launch_pack(const PackParams &p, vr_dtype dtype, cudaStream_t s)
{
    if (p.count <= 0) return cudaSuccess;
    const int threads = 256;
    long long blocks = (p.count + threads - 1) / threads;
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
    const size_t smem = static_cast<size_t>(p.ntf) * sizeof(float4);
#define VR_MARCH(T)                                                                      \
    (count ? (march_kernel<T, true><<<p.n_items, 128, smem, s>>>(p), 0)                  \
           : (march_kernel<T, false><<<p.n_items, 128, smem, s>>>(p), 0))
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
