// vr_staged.cu -- the per-brick march with brick data staged in shared memory
// (an alternative to the xy-quad march of vr_kernels.cu, selected with
// vr_set_march_staging).
//
// Sec. 2.2 of arXiv:2501.01628: each rank renders the share of the data it
// holds. Here one block marches the rays of one 8x16-pixel tile of a brick's
// footprint, slab by slab in depth: for each slab (up to 8 lattice samples of
// every ray of the tile) the box of brick voxels those samples can touch is
// copied from a scalar (one value per voxel) copy of the brick into shared
// memory with bulk asynchronous copies (cp.async.bulk, one per box row,
// completing on an mbarrier), while the block samples the previous slab from
// the other of two stages. The arithmetic of a sample -- position, floors,
// weights, the trilinear lerps, classification and accumulation -- is the
// quad march's, term for term, so both give the same image bit for bit.
//
// The box of a slab comes from the tile's four corner rays at the slab's two
// ends (one lattice step wider on each side, for the rounding of the per-ray
// sample ranges), widened by the spherical cap between them and one voxel.
// A slab of fewer samples is used when the box would not fit a stage; when not
// even one sample's box fits, the block samples that slab straight from the
// scalar brick in global memory.
//
// Every wait is bounded: a wait that gives up sets bit 5 (value 32) of the
// device error word (vr_sync reports VR_ERR_TIMEOUT), and the block stops after
// waiting, again bounded, for its copies in flight.
#include "vr_device.cuh"

namespace vr {
namespace {

using dev::over;

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase of `bar` with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int limit)
{
    for (int i = 0; i < limit; ++i) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred P;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, P;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_copy(float *dst, const float *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Box of haloed-local voxels [x0, x0+nx) x [y0, y0+ny) x [z0, z0+nz) staged for
// one slab (x0 and nx multiples of 4: 16-byte rows), and the slab's depth range.
struct Slab {
    float t0, t1;  // lattice samples with t in [t0, t1) (per-ray integer ranges)
    int x0, y0, z0, nx, ny, nz;
    bool staged;   // false: sampled straight from global memory
};

constexpr int kWaitLimit = 1 << 22;

template <bool COUNT, bool OPC>
__global__ void __launch_bounds__(128) march_staged_kernel(const __grid_constant__ MarchParams p,
                                                           const __grid_constant__ StagedBricks sb)
{
    extern __shared__ __align__(128) float stage[];  // [2][kStageCap]
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ float red[2][4];
    asm volatile("griddepcontrol.launch_dependents;");
    if (static_cast<int>(blockIdx.x) < p.mask_blocks) {  // the composite's tile masks
        dev::write_tile_mask(blockIdx.x * kMaskThreads + threadIdx.x, p.mask_tiles_x, p.mask_tiles_y, p.nb, p.order,
                             [&](int b) {
                                 return make_int4(p.b[b].rect[0], p.b[b].rect[1], p.b[b].rect[2], p.b[b].rect[3]);
                             },
                             p.tile_mask);
        return;
    }
    const int tid = threadIdx.x;
    const int item = blockIdx.x - p.mask_blocks;
    const int bi = dev::find_brick(p, item);
    const BrickLaunch &B = p.b[bi];
    const int local = item - B.item_begin;
    const int ty = local / B.tiles_x, tx = local - ty * B.tiles_x;
    const int warp = tid >> 5, lane = tid & 31;
    const int rx = tx * p.tile_w + (warp & 1) * p.pw + (lane & (p.pw - 1));
    const int ry = ty * p.tile_h + (warp >> 1) * (32 / p.pw) + lane / p.pw;
    const bool in_rect = rx < B.rect[2] && ry < B.rect[3];
    const int sx = B.sx, sy = B.sy, sz = B.hi[2] - B.lo[2] + 2;  // haloed extents
    const int sxp = sb.sxp[bi];
    const float *vox = sb.scalar + sb.sbase[bi];

    // this thread's ray and owned run
    dev::Ray ray;
    dev::OwnedRun run;
    run.ka = 0;
    run.kb = -1;
    if (in_rect) {
        dev::ray_setup(p, B.rect[0] + rx, B.rect[1] + ry, ray);
        dev::brick_run(p, B, ray, run);
    }
    const bool has_run = run.ka <= run.kb;
    // the tile's depth range: block min of t(ka), max of t(kb)
    float tlo = has_run ? fmaf(static_cast<float>(run.ka) + 0.5f, p.dt, ray.t_in) : 3.0e38f;
    float thi = has_run ? fmaf(static_cast<float>(run.kb) + 0.5f, p.dt, ray.t_in) : -3.0e38f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tlo = fminf(tlo, __shfl_xor_sync(0xffffffffu, tlo, o));
        thi = fmaxf(thi, __shfl_xor_sync(0xffffffffu, thi, o));
    }
    if (lane == 0) {
        red[0][warp] = tlo;
        red[1][warp] = thi;
    }
    if (tid == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    tlo = fminf(fminf(red[0][0], red[0][1]), fminf(red[0][2], red[0][3]));
    thi = fmaxf(fmaxf(red[1][0], red[1][1]), fmaxf(red[1][2], red[1][3]));

    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
    unsigned long long executed = 0;
    if (tlo <= thi) {  // the block has samples (uniform)
        // corner rays of the tile (the same for every thread)
        const int cx0 = B.rect[0] + tx * p.tile_w, cy0 = B.rect[1] + ty * p.tile_h;
        const int cx1 = min(cx0 + p.tile_w, B.rect[0] + B.rect[2]) - 1;
        const int cy1 = min(cy0 + p.tile_h, B.rect[1] + B.rect[3]) - 1;
        dev::Ray cr[4];
        dev::ray_setup(p, cx0, cy0, cr[0]);
        dev::ray_setup(p, cx1, cy0, cr[1]);
        dev::ray_setup(p, cx0, cy1, cr[2]);
        dev::ray_setup(p, cx1, cy1, cr[3]);
        // spherical-cap bound: a tile ray lies within t (1 - cos theta) of the
        // corners' hull at distance t, theta the widest corner angle from their mean
        float cap = 0.0f;
        if (!p.ortho) {
            float m[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) m[a] = cr[0].dv[a] + cr[1].dv[a] + cr[2].dv[a] + cr[3].dv[a];
            const float mn = rsqrtf(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
            float cmin = 1.0f;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                cmin = fminf(cmin, (cr[c].dv[0] * m[0] + cr[c].dv[1] * m[1] + cr[c].dv[2] * m[2]) * mn / p.nmax);
            cap = 1.0f - cmin;
        }
        const float shift[3] = {static_cast<float>(B.lo[0]) - 0.5f, static_cast<float>(B.lo[1]) - 0.5f,
                                static_cast<float>(B.lo[2]) - 0.5f};
        // the box of samples with t in [t0, t1): corners at t0 - dt and t1 + dt
        auto box = [&](float t0, float t1, Slab &sl) {
            const float ta = t0 - p.dt, tb = t1 + p.dt;
            const float margin = 1.0f + fmaxf(fabsf(ta), fabsf(tb)) * p.nmax * cap;
            float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float va = fmaf(ta, cr[c].dv[a], cr[c].ov[a]) - shift[a];
                    const float vb = fmaf(tb, cr[c].dv[a], cr[c].ov[a]) - shift[a];
                    lo[a] = fminf(lo[a], fminf(va, vb));
                    hi[a] = fmaxf(hi[a], fmaxf(va, vb));
                }
            const int ext[3] = {sx, sy, sz};
            int b0[3], b1[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                // [b0, b1) with at least two voxels on every axis, inside the brick
                b0[a] = min(max(0, static_cast<int>(floorf(fmaxf(lo[a] - margin, -1.0f)))), ext[a] - 2);
                b1[a] = max(min(ext[a], static_cast<int>(floorf(fminf(hi[a] + margin, 1.0e6f))) + 2), b0[a] + 2);
            }
            sl.t0 = t0;
            sl.t1 = t1;
            sl.x0 = b0[0] & ~3;
            sl.nx = min((b1[0] + 3) & ~3, sxp) - sl.x0;
            sl.y0 = b0[1];
            sl.ny = b1[1] - b0[1];
            sl.z0 = b0[2];
            sl.nz = b1[2] - b0[2];
            return sl.nx * sl.ny * sl.nz <= kStageCap;
        };
        // the next slab from t0: 8 samples, fewer when the box does not fit
        auto plan = [&](float t0, Slab &sl) {
            if (!(t0 + p.dt > t0)) {  // a step below the rounding of t: one last slab from global memory
                sl.t0 = t0;
                sl.t1 = 3.0e38f;
                sl.staged = false;
                return;
            }
            for (int n = 8; n >= 1; n >>= 1)
                if (box(t0, t0 + n * p.dt, sl)) {
                    sl.staged = true;
                    return;
                }
            sl.staged = false;
            sl.t1 = t0 + p.dt;
        };
        auto issue = [&](const Slab &sl, int st) {
            // generic-proxy reads of this stage (two slabs back) are ordered
            // before the async-proxy writes by the barrier above and this fence
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            float *dst = stage + st * kStageCap;
            const int rows = sl.ny * sl.nz;
            for (int r = tid; r < rows; r += 128) {
                const int zz = r / sl.ny, yy = r - zz * sl.ny;
                const float *src = vox + (static_cast<long long>(sl.z0 + zz) * sy + (sl.y0 + yy)) * sxp + sl.x0;
                bulk_copy(dst + r * sl.nx, src, static_cast<unsigned>(sl.nx) * 4u, &bar[st]);
            }
        };

        const float xmax = static_cast<float>(p.ntf - 1);
        const uintptr_t tf_base = reinterpret_cast<uintptr_t>(p.tf) - static_cast<uintptr_t>(dev::kFloorBits) * 32u;
        int kcur = run.ka;  // next sample of this thread's ray
        bool alive = has_run;
        unsigned phase = 0;  // bit s: parity of stage s's next phase
        bool failed = false;
        Slab cur, nxt;
        plan(tlo, cur);
        if (cur.staged) {
            if (tid == 0) mbar_expect_tx(&bar[0], static_cast<unsigned>(cur.nx * cur.ny * cur.nz) * 4u);
            __syncthreads();
            issue(cur, 0);
        }
        int st = 0;
        bool pending = cur.staged;  // stage st has copies in flight
        for (;;) {
            const bool last = cur.t1 > thi;
            // every thread is done with the stage the next slab reuses
            const bool any = __syncthreads_or(alive && kcur <= run.kb) != 0;
            const bool fail_any = __syncthreads_or(failed) != 0;  // the same decision in every thread
            if (!any || fail_any) break;
            if (!last) {
                plan(cur.t1, nxt);
                if (nxt.staged && tid == 0)
                    mbar_expect_tx(&bar[st ^ 1], static_cast<unsigned>(nxt.nx * nxt.ny * nxt.nz) * 4u);
                __syncthreads();
                if (nxt.staged) issue(nxt, st ^ 1);
            }
            if (cur.staged) {
                if (!mbar_wait(&bar[st], (phase >> st) & 1u, kWaitLimit)) {
                    if (tid == 0) atomicOr(p.count_error, 32);
                    failed = true;
                }
                phase ^= 1u << st;
                pending = false;
            }
            if (!failed && alive) {
                // this ray's samples of the slab: t_k in [t0, t1) by the lattice formula
                const int kend = last ? run.kb + 1
                                      : min(run.kb + 1, max(kcur, static_cast<int>(ceilf(
                                                                      (cur.t1 - ray.t_in) * p.inv_dt - 0.5f))));
                const float *sbuf = stage + st * kStageCap;
                const int nxy = cur.nx * cur.ny;
                float kh = static_cast<float>(kcur) + 0.5f;
                for (int k = kcur; k < kend; ++k, kh += 1.0f) {
                    const float vx = fmaf(kh, run.step[0], run.base[0]);
                    const float vy = fmaf(kh, run.step[1], run.base[1]);
                    const float vz = fmaf(kh, run.step[2], run.base[2]);
                    const float fx = floorf(vx), fy = floorf(vy), fz = floorf(vz);
                    const float wx = vx - fx, wy = vy - fy, wz = vz - fz;
                    const int ix = static_cast<int>(fx), iy = static_cast<int>(fy), iz = static_cast<int>(fz);
                    float v000, v100, v010, v110, v001, v101, v011, v111;
                    if (cur.staged) {
                        // the box holds the cell; the clamps only guard memory
                        const int lx = ix - cur.x0, ly = iy - cur.y0, lz = iz - cur.z0;
                        if (COUNT && (lx < 0 || lx + 1 >= cur.nx || ly < 0 || ly + 1 >= cur.ny || lz < 0 ||
                                      lz + 1 >= cur.nz))
                            atomicOr(p.count_error, 16);
                        const int i = min(max(lz, 0), cur.nz - 2) * nxy + min(max(ly, 0), cur.ny - 2) * cur.nx +
                                      min(max(lx, 0), cur.nx - 2);
                        v000 = sbuf[i];
                        v100 = sbuf[i + 1];
                        v010 = sbuf[i + cur.nx];
                        v110 = sbuf[i + cur.nx + 1];
                        v001 = sbuf[i + nxy];
                        v101 = sbuf[i + nxy + 1];
                        v011 = sbuf[i + nxy + cur.nx];
                        v111 = sbuf[i + nxy + cur.nx + 1];
                    } else {
                        const int cx = min(max(ix, 0), sx - 2), cy = min(max(iy, 0), sy - 2),
                                  cz = min(max(iz, 0), sz - 2);
                        const float *g = vox + (static_cast<long long>(cz) * sy + cy) * sxp + cx;
                        v000 = __ldg(g);
                        v100 = __ldg(g + 1);
                        v010 = __ldg(g + sxp);
                        v110 = __ldg(g + sxp + 1);
                        const float *g1 = g + static_cast<long long>(sy) * sxp;
                        v001 = __ldg(g1);
                        v101 = __ldg(g1 + 1);
                        v011 = __ldg(g1 + sxp);
                        v111 = __ldg(g1 + sxp + 1);
                    }
                    // the quad march's lerps, in its order
                    const float c00 = fmaf(wx, v100 - v000, v000), c10 = fmaf(wx, v110 - v010, v010);
                    const float c01 = fmaf(wx, v101 - v001, v001), c11 = fmaf(wx, v111 - v011, v011);
                    const float c0_ = fmaf(wy, c10 - c00, c00), c1_ = fmaf(wy, c11 - c01, c01);
                    const float s = fmaf(wz, c1_ - c0_, c0_);
                    float x = fmaf(s, p.tf_scale, p.tf_bias);
                    x = fminf(fmaxf(x, 0.0f), xmax);
                    const float y = __fadd_rd(x, dev::kFloorOffset);
                    const float w = x - (y - dev::kFloorOffset);
                    float4 e0, de;
                    dev::ldg_v8(reinterpret_cast<const float4 *>(tf_base +
                                                                 static_cast<uintptr_t>(__float_as_uint(y)) * 32u),
                                e0, de);
                    const float r = fmaf(w, de.x, e0.x), g = fmaf(w, de.y, e0.y), bb = fmaf(w, de.z, e0.z);
                    float al = fmaf(w, de.w, e0.w);
                    if (OPC) al = -expm1f(p.opc_ratio * log1pf(-al));
                    const float ta = T * al;
                    C0 = fmaf(ta, r, C0);
                    C1 = fmaf(ta, g, C1);
                    C2 = fmaf(ta, bb, C2);
                    T = T - ta;
                    if (COUNT) ++executed;
                    if (T <= p.ert_T) {
                        alive = false;
                        break;
                    }
                }
                kcur = kend;
            }
            if (last) break;
            cur = nxt;
            st ^= 1;
            pending = cur.staged;
        }
        // nothing may be in flight into shared memory when the block exits
        if (pending && !mbar_wait(&bar[st], (phase >> st) & 1u, kWaitLimit) && tid == 0)
            atomicOr(p.count_error, 32);
    }
    if (in_rect) {
        float4 *dst = p.partials + B.poff + static_cast<long long>(ry) * B.rect[2] + rx;
        unsigned long long policy;
        asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(policy));
        asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(dst), "f"(C0), "f"(C1),
                     "f"(C2), "f"(1.0f - T), "l"(policy)
                     : "memory");
    }
    if (COUNT && executed) atomicAdd(p.sample_counter, executed);
}

// Scalar copy of every brick: haloed (bx+2)(by+2)(bz+2) voxels, rows padded to
// a multiple of 4 (16 bytes), edge-clamped halo. One launch for all bricks; a
// block writes kPackChunk consecutive elements of one brick.
__global__ void __launch_bounds__(256) scalar_pack_kernel(const __grid_constant__ PackParams p)
{
    int lo = 0, hi = p.nb - 1;
    const int blk = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.b[mid].block_begin <= blk) lo = mid;
        else hi = mid - 1;
    }
    const PackBrick &B = p.b[lo];
    float *dst = static_cast<float *>(B.dst);
    const int row = B.row;
    const long long e0 = static_cast<long long>(blk - B.block_begin) * kPackChunk;
    const long long e1 = min(e0 + kPackChunk, B.quads);
    for (long long e = e0 + threadIdx.x; e < e1; e += 256) {
        const int lx = static_cast<int>(e % row);
        const long long rest = e / row;
        const int ly = static_cast<int>(rest % B.s[1]);
        const int lz = static_cast<int>(rest / B.s[1]);
        const int gx = min(max(B.lo[0] + lx - 1, 0), p.N[0] - 1);
        const int gy = min(max(B.lo[1] + ly - 1, 0), p.N[1] - 1);
        const int gz = min(max(B.lo[2] + lz - 1, 0), p.N[2] - 1);
        dst[e] = __ldg(p.src + (static_cast<long long>(gz) * p.N[1] + gy) * p.N[0] + gx);
    }
}

}  // namespace

cudaError_t launch_march_staged(const MarchParams &p, const StagedBricks &sb, cudaStream_t s)
{
    const int grid = p.n_items + p.mask_blocks;
    if (grid <= 0) return cudaSuccess;
    constexpr size_t smem = 2 * kStageCap * sizeof(float);
    const bool count = p.sample_counter != nullptr;
    const bool opc = p.opc_ratio != 1.0f;
    if (opc) {
        if (count) march_staged_kernel<true, true><<<grid, 128, smem, s>>>(p, sb);
        else march_staged_kernel<false, true><<<grid, 128, smem, s>>>(p, sb);
    } else {
        if (count) march_staged_kernel<true, false><<<grid, 128, smem, s>>>(p, sb);
        else march_staged_kernel<false, false><<<grid, 128, smem, s>>>(p, sb);
    }
    return cudaGetLastError();
}

cudaError_t launch_scalar_pack(const PackParams &p, cudaStream_t s)
{
    if (p.n_blocks <= 0) return cudaSuccess;
    scalar_pack_kernel<<<p.n_blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace vr
