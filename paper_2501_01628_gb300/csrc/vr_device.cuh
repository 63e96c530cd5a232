// vr_device.cuh -- device code shared by the forward kernels (vr_kernels.cu)
// and the adjoint kernels (vr_grad.cu): brick storage loads, work-item lookup,
// and the per-ray, per-brick sample run.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "vr_internal.h"

namespace vr {
namespace dev {

// ---------------------------------------------------------------------------
// Brick storage: "xy-quads". Element (i,j,k) of a brick whose haloed extents
// are (sx, sy, sz) holds the four voxels (i,j,k), (i+1,j,k), (i,j+1,k),
// (i+1,j+1,k), for i < sx-1, j < sy-1, k < sz. A trilinear sample then needs
// two vector loads (planes k and k+1) instead of eight scalar gathers, at four
// times the storage -- L1 wavefronts, not HBM capacity, bound the march.
// ---------------------------------------------------------------------------
template <typename T> struct Quad;
template <> struct Quad<float> {
    static constexpr bool octet = false;
    using type = float4;
    static __device__ __forceinline__ float4 load(const float4 *p) { return __ldg(p); }
    static __device__ __forceinline__ float4 make(float a, float b, float c, float d)
    {
        return make_float4(a, b, c, d);
    }
};
template <> struct Quad<__nv_bfloat16> {
    static constexpr bool octet = false;
    using type = uint2;
    static __device__ __forceinline__ float4 load_bits(uint2 u)
    {
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                           __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
    }
    static __device__ __forceinline__ float4 load(const uint2 *p) { return load_bits(__ldg(p)); }
    static __device__ __forceinline__ uint2 make(float a, float b, float c, float d)
    {
        auto bits = [](float v) {
            return static_cast<unsigned>(__bfloat16_as_ushort(__float2bfloat16_rn(v)));
        };
        return make_uint2(bits(a) | (bits(b) << 16), bits(c) | (bits(d) << 16));
    }
};
template <> struct Quad<__half> {
    static constexpr bool octet = false;
    using type = uint2;
    static __device__ __forceinline__ float4 load_bits(uint2 u)
    {
        const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
        const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    }
    static __device__ __forceinline__ float4 load(const uint2 *p) { return load_bits(__ldg(p)); }
    static __device__ __forceinline__ uint2 make(float a, float b, float c, float d)
    {
        auto bits = [](float v) { return static_cast<unsigned>(__half_as_ushort(__float2half_rn(v))); };
        return make_uint2(bits(a) | (bits(b) << 16), bits(c) | (bits(d) << 16));
    }
};

// "Octets": 16-bit storage with both planes of a cell in one 16-byte element,
// (plane k quad, plane k+1 quad), at the quad's index. A sample is then one
// 128-bit load; the storage is twice that of 16-bit xy-quads (the same as
// float32 xy-quads). Octet<T> tags the layout in the kernels' templates.
template <typename T> struct Octet {};
template <typename T> struct OctetOf {
    static constexpr bool octet = true;
    using type = uint4;
    static __device__ __forceinline__ void load2(const uint4 *p, float4 &a0, float4 &a1)
    {
        const uint4 u = __ldg(p);
        a0 = Quad<T>::load_bits(make_uint2(u.x, u.y));
        a1 = Quad<T>::load_bits(make_uint2(u.z, u.w));
    }
    static __device__ __forceinline__ uint4 make8(float a, float b, float c, float d, float e, float f, float g,
                                                  float h)
    {
        const uint2 lo = Quad<T>::make(a, b, c, d), hi = Quad<T>::make(e, f, g, h);
        return make_uint4(lo.x, lo.y, hi.x, hi.y);
    }
};
template <> struct Quad<Octet<__nv_bfloat16>> : OctetOf<__nv_bfloat16> {};
template <> struct Quad<Octet<__half>> : OctetOf<__half> {};

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

// The samples one brick owns along one pixel's ray, with the local
// voxel-centre coordinates of sample k: v = base + (k + 1/2) * step, where
// v = q - lo + 1/2 and q is the position in voxel units. Empty if ka > kb.
struct OwnedRun {
    float base[3], step[3];
    int ka, kb;
};

// A pixel's primary ray in voxel units, its whole-volume interval [t_in, t_out)
// and the rounding margin used for every brick's slab estimate. FP32, with the
// same arithmetic for every brick, so that each lattice sample has one owner.
struct Ray {
    float ov[3], dv[3], inv[3];
    float t_in, t_out;
    int margin;
    bool hit;
};

template <typename P>
__device__ __forceinline__ void ray_setup(const P &p, int px, int py, Ray &ray)
{
    const float fx = (static_cast<float>(px) + 0.5f) * p.inv_W;
    const float fy = (static_cast<float>(py) + 0.5f) * p.inv_H;
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
        const float inv = __frsqrt_rn(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
        for (int i = 0; i < 3; ++i) d[i] *= inv;
    }
    // voxel-space origin and direction; t stays in world units
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ray.ov[i] = o[i] * p.nmax;
        ray.dv[i] = d[i] * p.nmax;
    }
    // whole-volume interval (uses only (0 - o)/d and (N - o)/d)
    float t0 = 0.0f, t1 = 3.0e38f, dmin = 3.0e38f;
    bool hit = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (ray.dv[i] == 0.0f) {
            ray.inv[i] = 0.0f;
            if (ray.ov[i] < 0.0f || ray.ov[i] > p.N[i]) hit = false;
        } else {
            const float inv = __frcp_rn(ray.dv[i]);
            ray.inv[i] = inv;
            const float ta = (0.0f - ray.ov[i]) * inv, tb = (p.N[i] - ray.ov[i]) * inv;
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
            dmin = fminf(dmin, fabsf(ray.dv[i]));
        }
    }
    ray.t_in = t0;
    ray.t_out = t1;
    ray.hit = hit && t0 < t1;
    // slab estimates are widened by a margin covering FP32 rounding of the
    // positions (large only for rays nearly parallel to a face)
    ray.margin = 2 + static_cast<int>(fminf(1.0e6f, __fdividef(1.0e-6f * p.nmax, dmin * p.dt)));
}

// The samples brick B owns along `ray`: the slab estimate, made exact with the
// ownership test itself (sample k is owned iff it lies before t_out and its cell
// is in the brick).
template <typename P>
__device__ __forceinline__ void brick_run(const P &p, const BrickLaunch &B, const Ray &ray, OwnedRun &run)
{
    run.ka = 0;
    run.kb = -1;
    if (!ray.hit) return;
    float b0 = 0.0f, b1 = 3.0e38f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (ray.dv[i] == 0.0f) {
            if (ray.ov[i] < static_cast<float>(B.lo[i]) || ray.ov[i] > static_cast<float>(B.hi[i])) return;
        } else {
            const float ta = (static_cast<float>(B.lo[i]) - ray.ov[i]) * ray.inv[i];
            const float tb = (static_cast<float>(B.hi[i]) - ray.ov[i]) * ray.inv[i];
            b0 = fmaxf(b0, fminf(ta, tb));
            b1 = fminf(b1, fmaxf(ta, tb));
        }
    }
    if (!(b0 <= b1)) return;
    const float t_in = ray.t_in, t_out = ray.t_out;
    int ka = max(0, static_cast<int>(floorf((b0 - t_in) * p.inv_dt - 0.5f)) - ray.margin);
    int kb = static_cast<int>(ceilf((fminf(b1, t_out) - t_in) * p.inv_dt - 0.5f)) + ray.margin;
    auto owned = [&](int k) {
        const float t = fmaf(static_cast<float>(k) + 0.5f, p.dt, t_in);
        const float qxv = fmaf(t, ray.dv[0], ray.ov[0]);
        const float qyv = fmaf(t, ray.dv[1], ray.ov[1]);
        const float qzv = fmaf(t, ray.dv[2], ray.ov[2]);
        return t < t_out && qxv >= B.own_lo[0] && qxv < B.own_hi[0] && qyv >= B.own_lo[1] && qyv < B.own_hi[1] &&
               qzv >= B.own_lo[2] && qzv < B.own_hi[2];
    };
    while (ka <= kb && !owned(ka)) ++ka;
    while (kb > ka && !owned(kb)) --kb;
    // owned samples are contiguous along the ray: [ka, kb] are all owned
    run.ka = ka;
    run.kb = kb;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        run.step[i] = ray.dv[i] * p.dt;
        run.base[i] = fmaf(t_in, ray.dv[i], ray.ov[i] - (static_cast<float>(B.lo[i]) - 0.5f));
    }
}

template <typename P>
__device__ __forceinline__ void owned_run(const P &p, const BrickLaunch &B, int px, int py, OwnedRun &run)
{
    Ray ray;
    ray_setup(p, px, py, ray);
    brick_run(p, B, ray, run);
}

// Packed FP32 pairs (sm_100 family): two lanes of one 64-bit register, each
// rounded as the scalar instruction would be.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// a + b rounded towards -infinity in both lanes
__device__ __forceinline__ unsigned long long f2_add_rm(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// floor by the 1.5 * 2^23 offset: for |v| < 2^22, y = v + 1.5 * 2^23 rounded
// towards -infinity is exactly 1.5 * 2^23 + floor(v), whose bit pattern is
// kFloorBits + floor(v) (the binade of y has unit spacing).
constexpr float kFloorOffset = 12582912.0f;
constexpr unsigned kFloorBits = 0x4B400000u;

// 32 bytes at a 32-byte aligned address in one 256-bit load (sm_100 and later)
__device__ __forceinline__ void ldg_v8(const float4 *p, float4 &a, float4 &b)
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// Pipelined frames: before a march block stores into its partial pool, the
// composite that last read the pool (frame pool_frame - 2) must be done with
// it; that composite publishes its frame number in pool_done[pool] with a
// release store once every one of its blocks has read its partials (CTA
// barrier, gpu-scope fence, counter). The order needed is write-after-read:
// the polling thread's stores are issued only after the polled value has
// arrived (they depend on it through the branch; stores are not performed
// speculatively), and the composite's loads had returned their data before it
// released the pool. The poll is therefore a relaxed load from L2: an acquire
// at gpu scope would also invalidate the SM's L1, which the co-resident march
// blocks live on (measured: 0.607 against 0.576 ms per pipelined frame). The
// loop is one opaque inline-PTX block, so it leaves the caller's code
// generation alone; after kPoolWaitPolls polls it sets bit 6 (value 64) of the
// error word and returns false (the caller then skips its stores).
constexpr int kPoolWaitPolls = 1 << 20;
__device__ __forceinline__ bool pool_ready(const unsigned long long *pool_done, int pool,
                                           unsigned long long frame, int *error)
{
    if (!pool_done || frame < 2) return true;
    unsigned ok;
    asm volatile(
        "{\n\t"
        ".reg .pred pd;\n\t"
        ".reg .u64 v;\n\t"
        ".reg .u32 n;\n\t"
        "mov.u32 n, 0;\n"
        "VR_POOL_POLL:\n\t"
        "ld.relaxed.gpu.global.u64 v, [%1];\n\t"
        "setp.ge.u64 pd, v, %2;\n\t"
        "@pd bra VR_POOL_OK;\n\t"
        "add.u32 n, n, 1;\n\t"
        "setp.ge.u32 pd, n, %3;\n\t"
        "@pd bra VR_POOL_FAIL;\n\t"
        "nanosleep.u32 64;\n\t"
        "bra VR_POOL_POLL;\n"
        "VR_POOL_FAIL:\n\t"
        "red.global.or.b32 [%4], 64;\n\t"
        "mov.u32 %0, 0;\n\t"
        "bra VR_POOL_END;\n"
        "VR_POOL_OK:\n\t"
        "mov.u32 %0, 1;\n"
        "VR_POOL_END:\n\t"
        "}"
        : "=r"(ok)
        : "l"(pool_done + pool), "l"(frame - 2), "r"(kPoolWaitPolls), "l"(error)
        : "memory");
    return ok != 0;
}

// Front-to-back emission-absorption over one owned run (see include/vr.h):
// C += T alpha rgb, T *= (1 - alpha), continuing from the state (C, T) passed
// in, and stopping once T <= ert_T.
//
// The samples go in pairs (k, k+1). The pair's positions, floors and weights
// are computed in packed FP32 lanes; floors use the 1.5 * 2^23 offset, so the
// floor's bit pattern gives the cell without a conversion. The quad index is
// the blocked layout's (quad_index) written as a sum of per-axis terms,
//   4i - 3(i&1) + 4 nbx j + (2 - 4 nbx)(j&1) + 4 nbx nby k + (4 - 4 nbx nby)(k&1),
// evaluated on the floors' bit patterns, and plane k+1's quad lies
// 4 + (k&1)(8 nbx nby - 8) further on; both are clamped to the brick's storage
// (owned samples always lie inside the brick, so the clamp only guards memory).
// Both cells' quads are requested before either sample is classified, a sample
// in the previous sample's cell reuses its quads, and both samples'
// transfer-function pairs are requested before the first is accumulated.
// OPC: opacity correction for a step other than the reference step,
// alpha' = 1 - (1 - alpha)^ratio, evaluated as -expm1(ratio * log1p(-alpha)).
template <typename S, bool COUNT, bool OPC = false>
__device__ __forceinline__ void march_accumulate(const void *data, const BrickLaunch &B, const OwnedRun &run,
                                                 const float4 *tf, float tf_scale, float tf_bias, int ntf,
                                                 float ert_T, float &C0, float &C1, float &C2, float &T,
                                                 unsigned long long &executed, float opc_ratio = 1.0f,
                                                 int *count_error = nullptr)
{
    const int ka = run.ka, kb = run.kb;
    if (ka > kb) return;
    using Q = typename Quad<S>::type;
    const Q *vox = static_cast<const Q *>(data) + B.base;
    const unsigned nbx = static_cast<unsigned>(B.sx / 2), nby = static_cast<unsigned>(B.sy / 2);
    const unsigned nbz = static_cast<unsigned>(B.hi[2] - B.lo[2] + 3) / 2;
    const unsigned last = nbx * nby * nbz * 8u - 1u;  // last quad of the brick's storage
    const unsigned ay = 4u * nbx, az = 4u * nbx * nby;
    const unsigned c0 = 0u - (4u + ay + az) * kFloorBits;  // removes the offsets' bits
    const unsigned py = 2u - ay, pz = 4u - az, dz = 2u * az - 8u;
    const float xmax = static_cast<float>(ntf - 1);
    // transfer-function pair i at tf + 2 i, addressed from the floor's bits
    const uintptr_t tf_base = reinterpret_cast<uintptr_t>(tf) - static_cast<uintptr_t>(kFloorBits) * 32u;
    const unsigned long long off2 = f2_pack(kFloorOffset, kFloorOffset);
    const unsigned long long st_x = f2_pack(run.step[0], run.step[0]), bs_x = f2_pack(run.base[0], run.base[0]);
    const unsigned long long st_y = f2_pack(run.step[1], run.step[1]), bs_y = f2_pack(run.base[1], run.base[1]);
    const unsigned long long st_z = f2_pack(run.step[2], run.step[2]), bs_z = f2_pack(run.base[2], run.base[2]);
    const unsigned long long tfs2 = f2_pack(tf_scale, tf_scale), tfb2 = f2_pack(tf_bias, tf_bias);
    // quad indices of the cell (plane k) and of plane k+1 from the floors' bits
    // the counting variant also checks the claim that the clamps only guard
    // memory: an owned sample's quads must lie in the brick's storage
    auto cells = [&](unsigned bx, unsigned by, unsigned bz, unsigned &cell, unsigned &cell1, bool owned) {
        unsigned c = bz * az + c0;
        c = by * ay + c;
        c = bx * 4u + c;
        c = (bx & 1u) * (0u - 3u) + c;
        c = (by & 1u) * py + c;
        c = (bz & 1u) * pz + c;
        const unsigned c1 = c + 4u + (bz & 1u) * dz;
        if (COUNT && owned && count_error && (c > last || c1 > last)) atomicOr(count_error, 16);
        cell1 = min(c1, last);
        cell = min(c, last);
    };
    auto trilinear = [&](const float4 &a0, const float4 &a1, float wx, float wy, float wz) {
        const float c00 = fmaf(wx, a0.y - a0.x, a0.x), c10 = fmaf(wx, a0.w - a0.z, a0.z);
        const float c01 = fmaf(wx, a1.y - a1.x, a1.x), c11 = fmaf(wx, a1.w - a1.z, a1.z);
        const float c0_ = fmaf(wy, c10 - c00, c00), c1_ = fmaf(wy, c11 - c01, c01);
        return fmaf(wz, c1_ - c0_, c0_);
    };
    auto accumulate = [&](const float4 &e0, const float4 &de, float w) {
        const float r = fmaf(w, de.x, e0.x), g = fmaf(w, de.y, e0.y);
        const float bb = fmaf(w, de.z, e0.z);
        float al = fmaf(w, de.w, e0.w);
        if (OPC) al = -expm1f(opc_ratio * log1pf(-al));
        const float ta = T * al;
        C0 = fmaf(ta, r, C0);
        C1 = fmaf(ta, g, C1);
        C2 = fmaf(ta, bb, C2);
        T = T - ta;
    };
    unsigned prev = 0xffffffffu;
    float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
    float kh = static_cast<float>(ka) + 0.5f;
    for (int k = ka; k <= kb; k += 2, kh += 2.0f) {
        const bool two = k < kb;
        // positions (voxel-centre coordinates) of samples k and k+1, their
        // floors (offset form) and weights
        const unsigned long long h2 = f2_pack(kh, kh + 1.0f);
        const unsigned long long vx = f2_fma(h2, st_x, bs_x), vy = f2_fma(h2, st_y, bs_y),
                                 vz = f2_fma(h2, st_z, bs_z);
        const unsigned long long yx = f2_add_rm(vx, off2), yy = f2_add_rm(vy, off2), yz = f2_add_rm(vz, off2);
        float ax, bx_, ay_, by_, az_, bz_;
        f2_unpack(f2_sub(vx, f2_sub(yx, off2)), ax, bx_);
        f2_unpack(f2_sub(vy, f2_sub(yy, off2)), ay_, by_);
        f2_unpack(f2_sub(vz, f2_sub(yz, off2)), az_, bz_);
        float fxa, fxb, fya, fyb, fza, fzb;
        f2_unpack(yx, fxa, fxb);
        f2_unpack(yy, fya, fyb);
        f2_unpack(yz, fza, fzb);
        unsigned ca, ca1, cb, cb1;
        cells(__float_as_uint(fxa), __float_as_uint(fya), __float_as_uint(fza), ca, ca1, true);
        cells(__float_as_uint(fxb), __float_as_uint(fyb), __float_as_uint(fzb), cb, cb1, two);
        float4 r0, r1;
        if constexpr (Quad<S>::octet) {  // both planes in one element
            if (ca != prev) Quad<S>::load2(vox + ca, q0, q1);
            r0 = q0;
            r1 = q1;
            if (two && cb != ca) Quad<S>::load2(vox + cb, r0, r1);
        } else {
            if (ca != prev) {
                q0 = Quad<S>::load(vox + ca);
                q1 = Quad<S>::load(vox + ca1);
            }
            r0 = q0;
            r1 = q1;
            if (two && cb != ca) {
                r0 = Quad<S>::load(vox + cb);
                r1 = Quad<S>::load(vox + cb1);
            }
        }
        // both samples' table coordinates x = clamp((s - vmin)/(vmax - vmin), 0, 1)(n - 1)
        const float sa = trilinear(q0, q1, ax, ay_, az_);
        const float sb = trilinear(r0, r1, bx_, by_, bz_);
        float xa, xb;
        f2_unpack(f2_fma(f2_pack(sa, sb), tfs2, tfb2), xa, xb);
        xa = fminf(fmaxf(xa, 0.0f), xmax);
        xb = fminf(fmaxf(xb, 0.0f), xmax);
        const unsigned long long x2 = f2_pack(xa, xb);
        const unsigned long long y2 = f2_add_rm(x2, off2);
        float wa, wb, ya, yb;
        f2_unpack(f2_sub(x2, f2_sub(y2, off2)), wa, wb);
        f2_unpack(y2, ya, yb);
        float4 ea, da, eb, db;
        ldg_v8(reinterpret_cast<const float4 *>(tf_base + static_cast<uintptr_t>(__float_as_uint(ya)) * 32u), ea, da);
        ldg_v8(reinterpret_cast<const float4 *>(tf_base + static_cast<uintptr_t>(__float_as_uint(yb)) * 32u), eb, db);
        accumulate(ea, da, wa);
        if (COUNT) ++executed;
        if (T <= ert_T || !two) break;
        accumulate(eb, db, wb);
        if (COUNT) ++executed;
        if (T <= ert_T) break;
        q0 = r0;
        q1 = r1;
        prev = cb;
    }
}

// One brick's partial from a fresh state: (C, 1 - T).
template <typename S, bool COUNT, bool OPC = false>
__device__ __forceinline__ float4 march_run(const void *data, const BrickLaunch &B, const OwnedRun &run,
                                            const float4 *tf, float tf_scale, float tf_bias, int ntf, float ert_T,
                                            unsigned long long &executed, float opc_ratio = 1.0f,
                                            int *count_error = nullptr)
{
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
    march_accumulate<S, COUNT, OPC>(data, B, run, tf, tf_scale, tf_bias, ntf, ert_T, C0, C1, C2, T, executed,
                                    opc_ratio, count_error);
    return make_float4(C0, C1, C2, 1.0f - T);
}

// ---------------------------------------------------------------------------
// Composite tile masks: one thread per composite tile (kCompW x kCompTileH
// pixels) sets bit j of its 128-bit mask when the brick at visibility position
// j has a non-empty footprint rectangle that overlaps the tile. Every thread
// walks the positions in the same order, so the rectangle reads are uniform
// across the warp (broadcast, not per-lane gathers).
// ---------------------------------------------------------------------------
template <typename RectOf>
__device__ __forceinline__ void write_tile_mask(int tile, int tiles_x, int tiles_y, int nb, const int *order,
                                                RectOf rect_of, uint4 *mask)
{
    if (tile >= tiles_x * tiles_y) return;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int x0 = tx * kCompW, y0 = ty * kCompTileH;
    unsigned long long lo = 0, hi = 0;
    for (int j = 0; j < nb; ++j) {
        const int4 r = rect_of(order[j]);
        const bool ov = r.z > 0 && r.w > 0 && r.x < x0 + kCompW && x0 < r.x + r.z && r.y < y0 + kCompTileH &&
                        y0 < r.y + r.w;
        if (ov) {
            if (j < 64) lo |= 1ull << j;
            else hi |= 1ull << (j - 64);
        }
    }
    mask[tile] = make_uint4(static_cast<unsigned>(lo), static_cast<unsigned>(lo >> 32), static_cast<unsigned>(hi),
                            static_cast<unsigned>(hi >> 32));
}

__device__ __forceinline__ float4 over(float4 front, float4 back)
{
    const float w = 1.0f - front.w;
    return make_float4(fmaf(w, back.x, front.x), fmaf(w, back.y, front.y), fmaf(w, back.z, front.z),
                       fmaf(w, back.w, front.w));
}

}  // namespace dev
}  // namespace vr
