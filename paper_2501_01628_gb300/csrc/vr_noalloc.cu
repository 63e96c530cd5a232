// vr_noalloc.cu -- vr_render_frame_noalloc: a whole frame (per-brick march +
// composite) that allocates no device memory.
//
// Who needs it: a renderer embedded in another program's GPU job -- an
// in-situ plugin inside a simulation that hands all device memory to its own
// pool allocator, or a caller on a latency-critical path where cudaMalloc and
// cudaFree (which synchronise the device) are not allowed. Such a caller owns
// the volume, the output image and the stream; the library supplies only the
// scratch: the per-brick partial images and the transfer-function table, kept in
// one file-scope device array of fixed size, VR_NOALLOC_SCRATCH_BYTES.
//
// The arithmetic is the same as vr_render_frame's. The march reads the
// caller's x-fastest float32 volume directly (edge-clamped trilinear, eight
// scalar loads per sample) instead of the library's packed bricks, because
// packing would need device memory.
#include <cmath>
#include <cstring>
#include <vector>

#include "vr_internal.h"

namespace vr {
namespace {

// Scratch shared by every call on a device, held until the process exits:
// [0, kTfBytes) transfer-function pairs, then the composite's tile masks (one
// 16-byte mask per 32 x 8 tile of the image), then the partial images (float4).
constexpr size_t kScratchBytes = VR_NOALLOC_SCRATCH_BYTES;
constexpr size_t kTfBytes = 2 * 1024 * sizeof(float4);
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch on the current device. The host-side symbol is
// not a device address; the lookup is repeated on every call (it is cheap once
// the module is loaded), so a device reset or a re-created primary context
// never leaves a stale address behind.
cudaError_t scratch_address(void **out)
{
    *out = nullptr;
    return cudaGetSymbolAddress(out, g_scratch);
}

__device__ __forceinline__ int find_brick_g(const MarchParams &p, int item)
{
    int lo = 0, hi = p.nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.b[mid].item_begin <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// March over the caller's global volume (p.data: x-fastest float32 with
// extents p.N). Ray setup, lattice, ownership and accumulation as in the
// packed-brick march.
__global__ void __launch_bounds__(128) march_global_kernel(const __grid_constant__ MarchParams p)
{
    const int item = blockIdx.x;
    const BrickLaunch &B = p.b[find_brick_g(p, item)];
    const int local = item - B.item_begin;
    const int ty = local / B.tiles_x, tx = local - ty * B.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rx = tx * kTileW + (warp & 1) * 8 + (lane & 7);
    const int ry = ty * kTileH + (warp >> 1) * 4 + (lane >> 3);
    if (rx >= B.rect[2] || ry >= B.rect[3]) return;
    const int px = B.rect[0] + rx, py = B.rect[1] + ry;

    const float fx = (static_cast<float>(px) + 0.5f) * p.inv_W;
    const float fy = (static_cast<float>(py) + 0.5f) * p.inv_H;
    float o[3], d[3];
    if (p.ortho) {
        const float a = (fx - 0.5f) * p.ow, b = (fy - 0.5f) * p.oh;
        for (int i = 0; i < 3; ++i) {
            o[i] = fmaf(b, p.u[i], fmaf(a, p.r[i], p.eye[i]));
            d[i] = p.f[i];
        }
    } else {
        const float sx = (fx * 2.0f - 1.0f) * p.tanx, sy = (fy * 2.0f - 1.0f) * p.tany;
        for (int i = 0; i < 3; ++i) {
            o[i] = p.eye[i];
            d[i] = fmaf(sy, p.u[i], fmaf(sx, p.r[i], p.f[i]));
        }
        const float inv = __frsqrt_rn(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int i = 0; i < 3; ++i) d[i] *= inv;
    }
    float ov[3], dv[3];
    for (int i = 0; i < 3; ++i) {
        ov[i] = o[i] * p.nmax;
        dv[i] = d[i] * p.nmax;
    }
    float t0 = 0.0f, t1 = 3.0e38f, b0 = 0.0f, b1 = 3.0e38f;
    bool hit = true;
    for (int i = 0; i < 3; ++i) {
        if (dv[i] == 0.0f) {
            if (ov[i] < 0.0f || ov[i] > p.N[i]) hit = false;
            if (ov[i] < static_cast<float>(B.lo[i]) || ov[i] > static_cast<float>(B.hi[i])) hit = false;
        } else {
            const float inv = __frcp_rn(dv[i]);
            float ta = (0.0f - ov[i]) * inv, tb = (p.N[i] - ov[i]) * inv;
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
            ta = (static_cast<float>(B.lo[i]) - ov[i]) * inv;
            tb = (static_cast<float>(B.hi[i]) - ov[i]) * inv;
            b0 = fmaxf(b0, fminf(ta, tb));
            b1 = fminf(b1, fmaxf(ta, tb));
        }
    }
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
    if (hit && t0 < t1 && b0 <= b1) {
        const float t_in = t0, t_out = t1;
        float dmin = 3.0e38f;
        for (int i = 0; i < 3; ++i)
            if (dv[i] != 0.0f) dmin = fminf(dmin, fabsf(dv[i]));
        const int margin = 2 + static_cast<int>(fminf(1.0e6f, __fdividef(1.0e-6f * p.nmax, dmin * p.dt)));
        int ka = max(0, static_cast<int>(floorf((b0 - t_in) * p.inv_dt - 0.5f)) - margin);
        int kb = static_cast<int>(ceilf((fminf(b1, t_out) - t_in) * p.inv_dt - 0.5f)) + margin;
        auto owned = [&](int k) {
            const float t = fmaf(static_cast<float>(k) + 0.5f, p.dt, t_in);
            const float qxv = fmaf(t, dv[0], ov[0]);
            const float qyv = fmaf(t, dv[1], ov[1]);
            const float qzv = fmaf(t, dv[2], ov[2]);
            return t < t_out && qxv >= B.own_lo[0] && qxv < B.own_hi[0] && qyv >= B.own_lo[1] &&
                   qyv < B.own_hi[1] && qzv >= B.own_lo[2] && qzv < B.own_hi[2];
        };
        while (ka <= kb && !owned(ka)) ++ka;
        while (kb > ka && !owned(kb)) --kb;
        if (ka <= kb) {
            const float *vol = static_cast<const float *>(p.data);
            const int nx = static_cast<int>(p.N[0]), ny = static_cast<int>(p.N[1]), nz = static_cast<int>(p.N[2]);
            const float xmax = static_cast<float>(p.ntf - 1);
            float base[3], step[3];
            for (int i = 0; i < 3; ++i) {
                step[i] = dv[i] * p.dt;
                base[i] = fmaf(t_in, dv[i], ov[i] - 0.5f);  // global voxel-centre coordinates
            }
            float kh = static_cast<float>(ka) + 0.5f;
            for (int k = ka; k <= kb; ++k, kh += 1.0f) {
                const float vx = fmaf(kh, step[0], base[0]);
                const float vy = fmaf(kh, step[1], base[1]);
                const float vz = fmaf(kh, step[2], base[2]);
                const float flx = floorf(vx), fly = floorf(vy), flz = floorf(vz);
                const float wx = vx - flx, wy = vy - fly, wz = vz - flz;
                const int ix = static_cast<int>(flx), iy = static_cast<int>(fly), iz = static_cast<int>(flz);
                const int x0 = min(max(ix, 0), nx - 1), x1 = min(max(ix + 1, 0), nx - 1);
                const int y0 = min(max(iy, 0), ny - 1), y1 = min(max(iy + 1, 0), ny - 1);
                const int z0 = min(max(iz, 0), nz - 1), z1 = min(max(iz + 1, 0), nz - 1);
                const float *r00 = vol + (static_cast<long long>(z0) * ny + y0) * nx;
                const float *r10 = vol + (static_cast<long long>(z0) * ny + y1) * nx;
                const float *r01 = vol + (static_cast<long long>(z1) * ny + y0) * nx;
                const float *r11 = vol + (static_cast<long long>(z1) * ny + y1) * nx;
                const float v000 = __ldg(r00 + x0), v100 = __ldg(r00 + x1), v010 = __ldg(r10 + x0),
                            v110 = __ldg(r10 + x1), v001 = __ldg(r01 + x0), v101 = __ldg(r01 + x1),
                            v011 = __ldg(r11 + x0), v111 = __ldg(r11 + x1);
                const float c00 = fmaf(wx, v100 - v000, v000), c10 = fmaf(wx, v110 - v010, v010);
                const float c01 = fmaf(wx, v101 - v001, v001), c11 = fmaf(wx, v111 - v011, v011);
                const float c0 = fmaf(wy, c10 - c00, c00), c1 = fmaf(wy, c11 - c01, c01);
                const float s = fmaf(wz, c1 - c0, c0);
                const float x = fminf(fmaxf(fmaf(s, p.tf_scale, p.tf_bias), 0.0f), xmax);
                const int ti = static_cast<int>(x);
                const float w = x - static_cast<float>(ti);
                const float4 e0 = __ldg(p.tf + 2 * ti), de = __ldg(p.tf + 2 * ti + 1);
                const float ta = T * fmaf(w, de.w, e0.w);
                C0 = fmaf(ta, fmaf(w, de.x, e0.x), C0);
                C1 = fmaf(ta, fmaf(w, de.y, e0.y), C1);
                C2 = fmaf(ta, fmaf(w, de.z, e0.z), C2);
                T = T - ta;
                if (T <= p.ert_T) break;
            }
        }
    }
    p.partials[B.poff + static_cast<long long>(ry) * B.rect[2] + rx] = make_float4(C0, C1, C2, 1.0f - T);
}

bool normalize3(double v[3])
{
    const double l = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(l > 0.0)) return false;
    v[0] /= l;
    v[1] /= l;
    v[2] /= l;
    return true;
}

}  // namespace
}  // namespace vr

using namespace vr;

extern "C" vr_status vr_render_frame_noalloc(const float *volume_dev, const int dims[3], const vr_partition *part,
                                             const float *tf_rgba, int n_tf, float vmin, float vmax,
                                             const vr_camera *cam, float step_voxels, float ert_alpha,
                                             float *out_rgba_dev, void *stream)
{
    if (!volume_dev || !dims || !part || !tf_rgba || !cam || !out_rgba_dev) return VR_ERR_ARG;
    if (n_tf < 2 || n_tf > 1024 || !(vmax > vmin) || !(step_voxels > 0.0f) || !(ert_alpha > 0.0f))
        return VR_ERR_ARG;
    // host-side plan: bricks, front-to-back order and footprint rectangles
    int nb = 0;
    if (vr_partition_boxes(dims, part, &nb, nullptr) != VR_OK || nb < 1 || nb > kMaxBricks) return VR_ERR_ARG;
    std::vector<int> boxes(6 * static_cast<size_t>(nb)), order(nb), rects(4 * static_cast<size_t>(nb));
    vr_partition_boxes(dims, part, &nb, boxes.data());
    if (vr_plan_view(dims, part, cam, order.data(), rects.data()) != VR_OK) return VR_ERR_ARG;

    static thread_local MarchParams mp;
    std::memset(&mp, 0, sizeof(mp));
    long long px = 0;
    int items = 0;
    for (int b = 0; b < nb; ++b) {
        BrickLaunch &L = mp.b[b];
        const int *bx = &boxes[6 * b];
        const int *r = &rects[4 * b];
        for (int a = 0; a < 3; ++a) {
            L.lo[a] = bx[a];
            L.hi[a] = bx[3 + a];
            L.own_lo[a] = bx[a] == 0 ? -INFINITY : static_cast<float>(bx[a]);
            L.own_hi[a] = bx[3 + a] == dims[a] ? INFINITY : static_cast<float>(bx[3 + a]);
        }
        std::memcpy(L.rect, r, sizeof(L.rect));
        L.poff = px;
        px += static_cast<long long>(r[2]) * r[3];
        px = (px + 7) & ~7LL;
        L.item_begin = items;
        L.tiles_x = (r[2] + kTileW - 1) / kTileW;
        items += L.tiles_x * ((r[3] + kTileH - 1) / kTileH);
    }
    // the frame's partial images must fit the fixed scratch
    const int tiles_x = (cam->width + kCompW - 1) / kCompW, tiles_y = (cam->height + kCompTileH - 1) / kCompTileH;
    const size_t mask_bytes = static_cast<size_t>(tiles_x) * tiles_y * sizeof(uint4);
    if (static_cast<size_t>(px) * sizeof(float4) + mask_bytes > kScratchBytes - kTfBytes) return VR_ERR_ARG;

    double f[3] = {cam->dir[0], cam->dir[1], cam->dir[2]}, r[3], u[3];
    if (!normalize3(f)) return VR_ERR_ARG;
    r[0] = cam->up[1] * f[2] - cam->up[2] * f[1];
    r[1] = cam->up[2] * f[0] - cam->up[0] * f[2];
    r[2] = cam->up[0] * f[1] - cam->up[1] * f[0];
    if (!normalize3(r)) return VR_ERR_ARG;
    u[0] = f[1] * r[2] - f[2] * r[1];
    u[1] = f[2] * r[0] - f[0] * r[2];
    u[2] = f[0] * r[1] - f[1] * r[0];
    const double th = std::tan(cam->fovy_deg * M_PI / 360.0);
    const double nmax = std::max(dims[0], std::max(dims[1], dims[2]));
    for (int a = 0; a < 3; ++a) {
        mp.eye[a] = static_cast<float>(cam->eye[a]);
        mp.r[a] = static_cast<float>(r[a]);
        mp.u[a] = static_cast<float>(u[a]);
        mp.f[a] = static_cast<float>(f[a]);
        mp.N[a] = static_cast<float>(dims[a]);
    }
    mp.tany = static_cast<float>(th);
    mp.tanx = static_cast<float>(th * static_cast<double>(cam->width) / cam->height);
    mp.ow = static_cast<float>(cam->ortho_w);
    mp.oh = static_cast<float>(cam->ortho_h);
    mp.ortho = cam->ortho ? 1 : 0;
    mp.W = cam->width;
    mp.H = cam->height;
    mp.inv_W = static_cast<float>(1.0 / cam->width);
    mp.inv_H = static_cast<float>(1.0 / cam->height);
    mp.nmax = static_cast<float>(nmax);
    const double dt = static_cast<double>(step_voxels) / nmax;
    mp.dt = static_cast<float>(dt);
    mp.inv_dt = static_cast<float>(1.0 / dt);
    mp.ert_T = ert_alpha < 1.0f ? static_cast<float>(1.0 - static_cast<double>(ert_alpha)) : -1.0f;
    const double scale = (n_tf - 1) / (static_cast<double>(vmax) - vmin);
    mp.tf_scale = static_cast<float>(scale);
    mp.tf_bias = static_cast<float>(-static_cast<double>(vmin) * scale);
    mp.ntf = n_tf;
    mp.nb = nb;
    mp.n_items = items;
    mp.data = volume_dev;

    // transfer-function pairs (T[i], T[i+1] - T[i]), last difference 0
    std::vector<float> pairs(8 * static_cast<size_t>(n_tf));
    for (int i = 0; i < n_tf; ++i)
        for (int c = 0; c < 4; ++c) {
            const float a = tf_rgba[4 * i + c];
            const float b = i + 1 < n_tf ? tf_rgba[4 * (i + 1) + c] : a;
            pairs[8 * i + c] = a;
            pairs[8 * i + 4 + c] = b - a;
        }

    void *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess || !scratch) return VR_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float4 *tf_dev = static_cast<float4 *>(scratch);
    uint4 *masks = reinterpret_cast<uint4 *>(static_cast<unsigned char *>(scratch) + kTfBytes);
    float4 *partials = reinterpret_cast<float4 *>(static_cast<unsigned char *>(scratch) + kTfBytes + mask_bytes);
    // pageable source: the copy has left `pairs` before cudaMemcpyAsync returns
    if (cudaMemcpyAsync(tf_dev, pairs.data(), pairs.size() * sizeof(float), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return VR_ERR_CUDA;
    mp.tf = tf_dev;
    mp.partials = partials;
    if (items > 0) {
        march_global_kernel<<<items, 128, 0, s>>>(mp);
        if (cudaGetLastError() != cudaSuccess) return VR_ERR_CUDA;
    }
    // direct front-to-back composite with the existing kernel
    static thread_local CompositeParams cp;
    std::memset(&cp, 0, sizeof(cp));
    cp.W = cam->width;
    cp.H = cam->height;
    cp.nb = nb;
    cp.n_levels = 1;
    for (int j = 0; j < nb; ++j) cp.order[j] = order[j];
    for (int b = 0; b < nb; ++b) {
        std::memcpy(cp.rect[b], &rects[4 * b], 4 * sizeof(int));
        cp.poff[b] = mp.b[b].poff;
    }
    cp.partials = partials;
    cp.out = reinterpret_cast<float4 *>(out_rgba_dev);
    cp.tile_mask = masks;
    cp.tiles_x = tiles_x;
    cp.tiles_y = tiles_y;
    if (launch_tile_masks(cp, s) != cudaSuccess) return VR_ERR_CUDA;
    if (launch_composite(cp, s) != cudaSuccess) return VR_ERR_CUDA;
    return VR_OK;
}
