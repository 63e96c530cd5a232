// vr_mesh.cu -- march kernel (sm_103a) of tetrahedral-mesh volumes: the same
// per-brick emission-absorption runs on the global lattice as the voxel march
// (Sec. 2.2: each rank renders the samples of its share of the data), with the
// value taken from the brick's elements instead of a voxel grid.
//
// Per pixel and brick: the owned run [ka, kb] of lattice samples (ownership by
// the sample's cell, exactly as for voxel bricks), the element containing the
// first sample from a BVH point query, then a walk through face neighbours. In
// an element the value is linear in t and the ray leaves through the face whose
// barycentric coordinate falls to 0 first; every sample with t up to that exit
// parameter is classified and accumulated from the element's plane equation.
#include "vr_device.cuh"
#include "vr_mesh.h"

namespace vr {
namespace {

using dev::find_brick;
using dev::ldg_v8;

// Smallest barycentric coordinate of q in the element (record at rec).
__device__ __forceinline__ float min_bary(const float4 *rec, float qx, float qy, float qz)
{
    float4 r0, r1, r2, r3;
    ldg_v8(rec, r0, r1);
    ldg_v8(rec + 2, r2, r3);
    const float dx = qx - r0.x, dy = qy - r0.y, dz = qz - r0.z;
    const float l1 = fmaf(r1.x, dx, fmaf(r1.y, dy, fmaf(r1.z, dz, 0.25f)));
    const float l2 = fmaf(r2.x, dx, fmaf(r2.y, dy, fmaf(r2.z, dz, 0.25f)));
    const float l3 = fmaf(r3.x, dx, fmaf(r3.y, dy, fmaf(r3.z, dz, 0.25f)));
    const float l0 = 1.0f - l1 - l2 - l3;
    return fminf(fminf(l0, l1), fminf(l2, l3));
}

// Brick-local element containing q: a stackless preorder walk of the brick's
// BVH (node indices only increase), keeping the element with the largest
// smallest-barycentric among the leaves whose boxes hold q and stopping at the
// first element that holds q. Returns -1 only when no leaf box holds q.
__device__ int locate(const MeshParams &p, int brick, float qx, float qy, float qz)
{
    const MeshNode *nodes = p.nodes + p.node_base[brick];
    const float4 *rec = p.rec + kMeshRec * p.rec_base[brick];
    constexpr float eps = 1.0e-3f;  // voxel units
    int best = -1;
    float best_m = -3.0e38f;
    const int end = nodes[0].skip;
    int node = 0;
    while (node < end) {
        const MeshNode nd = nodes[node];
        const bool in = qx >= nd.lo[0] - eps && qx <= nd.hi[0] + eps && qy >= nd.lo[1] - eps &&
                        qy <= nd.hi[1] + eps && qz >= nd.lo[2] - eps && qz <= nd.hi[2] + eps;
        if (in && nd.leaf == 0) {
            ++node;
            continue;
        }
        if (in) {
            const int first = nd.leaf & ((1 << 28) - 1), count = nd.leaf >> 28;
            for (int i = 0; i < count; ++i) {
                const float m = min_bary(rec + kMeshRec * (first + i), qx, qy, qz);
                if (m > best_m) {
                    best_m = m;
                    best = first + i;
                }
            }
            if (best_m >= 0.0f) return best;
        }
        node = nd.skip;
    }
    return best;
}

// 8 blocks of 128 threads per SM: at most 64 registers per thread; a mask block
// writes one tile mask per thread
static_assert(kMaskThreads == 128, "mask blocks are march blocks");
template <bool COUNT, bool OPC>
__global__ void __launch_bounds__(128, 8) march_mesh_kernel(const __grid_constant__ MeshParams P)
{
    const MarchParams &p = P.m;
    // pipelined frames: the next grid may start once every block of this one
    // is running; the mask blocks write only after the preceding grid
    // completes, and the march blocks store their partials once the composite
    // that last read their pool is done (as in march_kernel); outside such
    // launches both waits return at once
    asm volatile("griddepcontrol.launch_dependents;");
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

    dev::Ray ray;
    dev::ray_setup(p, px, py, ray);
    dev::OwnedRun run;
    dev::brick_run(p, B, ray, run);
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, T = 1.f;
    unsigned long long executed = 0;
    if (run.ka <= run.kb) {
        const float4 *rec = P.rec + kMeshRec * P.rec_base[bi];
        const int4 *nbr = P.nbr + P.rec_base[bi];
        const float4 *tf = p.tf;
        const float xmax = static_cast<float>(p.ntf - 1);
        const float dvx = ray.dv[0], dvy = ray.dv[1], dvz = ray.dv[2];
        int k = run.ka;
        float t = fmaf(static_cast<float>(k) + 0.5f, p.dt, ray.t_in);
        float qx = fmaf(t, dvx, ray.ov[0]), qy = fmaf(t, dvy, ray.ov[1]), qz = fmaf(t, dvz, ray.ov[2]);
        int e = locate(P, bi, qx, qy, qz);
        if (e < 0) {
            atomicOr(P.error, 8);
            e = 0;
        }
        bool forced = true;  // a located element takes its first sample unconditionally
        int stall = 0;
        float4 r0, r1, r2, r3;
        ldg_v8(rec + kMeshRec * e, r0, r1);
        ldg_v8(rec + kMeshRec * e + 2, r2, r3);
        int4 nb = __ldg(nbr + e);
        // One element per iteration: every lane handles its current element
        // (the same instruction stream for the warp), requests the next
        // element's record, then takes the current element's samples while
        // that request is in flight.
        while (true) {
            // exit parameter: smallest t at which a decreasing barycentric
            // coordinate reaches 0, measured from the current sample position
            const float dx = qx - r0.x, dy = qy - r0.y, dz = qz - r0.z;
            const float n0x = -(r1.x + r2.x + r3.x), n0y = -(r1.y + r2.y + r3.y), n0z = -(r1.z + r2.z + r3.z);
            float t_exit = 3.0e38f;
            int face = -1;
            auto exit_face = [&](float nx, float ny, float nz, int f) {
                const float beta = fmaf(nx, dvx, fmaf(ny, dvy, nz * dvz));
                const float lam = fmaf(nx, dx, fmaf(ny, dy, fmaf(nz, dz, 0.25f)));
                const float tf_ = t - __fdividef(lam, beta);
                if (beta < 0.0f && tf_ < t_exit) {
                    t_exit = tf_;
                    face = f;
                }
            };
            exit_face(n0x, n0y, n0z, 0);
            exit_face(r1.x, r1.y, r1.z, 1);
            exit_face(r2.x, r2.y, r2.z, 2);
            exit_face(r3.x, r3.y, r3.z, 3);
            // value gradient g = sum_i (s_i - s_0) n_i; value(q) = s_mean + g . (q - c)
            const float gx = fmaf(r1.w, r1.x, fmaf(r2.w, r2.x, r3.w * r3.x));
            const float gy = fmaf(r1.w, r1.y, fmaf(r2.w, r2.y, r3.w * r3.y));
            const float gz = fmaf(r1.w, r1.z, fmaf(r2.w, r2.z, r3.w * r3.z));
            // the element after this one, requested before this one's samples
            int nx = face == 0 ? nb.x : face == 1 ? nb.y : face == 2 ? nb.z : face == 3 ? nb.w : -1;
            const int pe = nx >= 0 ? nx : e;
            const float4 *pr = rec + kMeshRec * pe;  // re-pointed after a locate
            float4 p0, p1, p2, p3;
            ldg_v8(pr, p0, p1);
            ldg_v8(pr + 2, p2, p3);
            int4 pn = __ldg(nbr + pe);
            bool done = false;
            while (forced || t <= t_exit) {
                forced = false;
                stall = 0;
                const float s = fmaf(gx, qx - r0.x, fmaf(gy, qy - r0.y, fmaf(gz, qz - r0.z, r0.w)));
                const float x = fminf(fmaxf(fmaf(s, p.tf_scale, p.tf_bias), 0.0f), xmax);
                const int ti = static_cast<int>(x);
                const float w = x - static_cast<float>(ti);
                float4 e0, de;
                ldg_v8(tf + 2 * ti, e0, de);
                float al = fmaf(w, de.w, e0.w);
                if (OPC) al = -expm1f(p.opc_ratio * log1pf(-al));
                const float ta = T * al;
                C0 = fmaf(ta, fmaf(w, de.x, e0.x), C0);
                C1 = fmaf(ta, fmaf(w, de.y, e0.y), C1);
                C2 = fmaf(ta, fmaf(w, de.z, e0.z), C2);
                T = T - ta;
                if (COUNT) ++executed;
                if (T <= p.ert_T || k >= run.kb) {
                    done = true;
                    break;
                }
                ++k;
                t = fmaf(static_cast<float>(k) + 0.5f, p.dt, ray.t_in);
                qx = fmaf(t, dvx, ray.ov[0]);
                qy = fmaf(t, dvy, ray.ov[1]);
                qz = fmaf(t, dvz, ray.ov[2]);
            }
            if (done) break;
            // the next sample lies beyond this element: the neighbour across the
            // exit face, or a new point location after a boundary face or too
            // many steps without a sample (rounding near edges and vertices)
            if (nx < 0 || ++stall > kMeshStallSteps) {
                nx = locate(P, bi, qx, qy, qz);
                if (nx < 0) {
                    atomicOr(P.error, 8);
                    nx = e;
                }
                forced = true;
                pr = rec + kMeshRec * nx;
                ldg_v8(pr, p0, p1);
                ldg_v8(pr + 2, p2, p3);
                pn = __ldg(nbr + nx);
            }
            e = nx;
            r0 = p0; r1 = p1; r2 = p2; r3 = p3;
            nb = pn;
        }
    }
    if (!dev::pool_ready(p.pool_done, p.pool, p.pool_frame, P.error)) return;
    p.partials[B.poff + static_cast<long long>(ry) * B.rect[2] + rx] = make_float4(C0, C1, C2, 1.0f - T);
    if (COUNT && executed) atomicAdd(p.sample_counter, executed);
}

}  // namespace

cudaError_t launch_march_mesh(const MeshParams &p, cudaStream_t s, bool after_frame)
{
    const int grid = p.m.n_items + p.m.mask_blocks;
    if (grid <= 0) return cudaSuccess;
    const bool count = p.m.sample_counter != nullptr, opc = p.m.opc_ratio != 1.0f;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(128);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = after_frame ? 1 : 0;
    if (count) return opc ? cudaLaunchKernelEx(&cfg, march_mesh_kernel<true, true>, p)
                          : cudaLaunchKernelEx(&cfg, march_mesh_kernel<true, false>, p);
    return opc ? cudaLaunchKernelEx(&cfg, march_mesh_kernel<false, true>, p)
               : cudaLaunchKernelEx(&cfg, march_mesh_kernel<false, false>, p);
}

}  // namespace vr
