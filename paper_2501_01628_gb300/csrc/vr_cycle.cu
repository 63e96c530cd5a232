// vr_cycle.cu -- CUDA kernel (sm_103a) of the ray-state cycling frame: one
// thread per pixel carries its ray's state through the bricks in visibility
// order (the ray-queue cycling of Sec. 2.2 and 3 of arXiv:2501.01628, restated
// for bricks on one GPU) and writes the final pixel; no partials, no composite.
#include <algorithm>

#include "vr_device.cuh"

namespace vr {
namespace {

// ---------------------------------------------------------------------------
// Ray-state cycling: one thread per image pixel carries (C, T) through the
// bricks in front-to-back order (the paper's ray-queue cycling, Sec. 2.2 and 3,
// where every ray visits every rank, restated for bricks on one GPU). No
// partial images and no composite; early termination is global.
// ---------------------------------------------------------------------------
template <typename S, bool COUNT, bool OPC>
__global__ void __launch_bounds__(128) march_cycle_kernel(const __grid_constant__ MarchParams p, float4 *out)
{
    // pipelined frames: the next frame's kernel may start once every block of
    // this grid is running, and this grid's image store waits for the
    // preceding grid (see march_kernel); outside such launches both are no-ops
    asm volatile("griddepcontrol.launch_dependents;");
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
    asm volatile("griddepcontrol.wait;" ::: "memory");
    out[static_cast<long long>(py) * p.W + px] = make_float4(C0, C1, C2, 1.0f - T);
    if (COUNT && executed) atomicAdd(p.sample_counter, executed);
}

}  // namespace

cudaError_t launch_march_cycle(const MarchParams &p, int kind, float4 *out, cudaStream_t s, bool after_frame)
{
    if (p.W <= 0 || p.H <= 0) return cudaSuccess;
    const dim3 grid((p.W + p.tile_w - 1) / p.tile_w, (p.H + p.tile_h - 1) / p.tile_h);
    const bool count = p.sample_counter != nullptr;
    const bool opc = p.opc_ratio != 1.0f;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(128);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = after_frame ? 1 : 0;
#define VR_CYCLE(T)                                                                                    \
    (opc ? (count ? cudaLaunchKernelEx(&cfg, march_cycle_kernel<T, true, true>, p, out)                \
                  : cudaLaunchKernelEx(&cfg, march_cycle_kernel<T, false, true>, p, out))              \
         : (count ? cudaLaunchKernelEx(&cfg, march_cycle_kernel<T, true, false>, p, out)               \
                  : cudaLaunchKernelEx(&cfg, march_cycle_kernel<T, false, false>, p, out)))
    cudaError_t e = cudaErrorInvalidValue;
    switch (kind) {
    case kStoreF32: e = VR_CYCLE(float); break;
    case kStoreBF16: e = VR_CYCLE(__nv_bfloat16); break;
    case kStoreF16: e = VR_CYCLE(__half); break;
    case kStoreBF16Oct: e = VR_CYCLE(dev::Octet<__nv_bfloat16>); break;
    case kStoreF16Oct: e = VR_CYCLE(dev::Octet<__half>); break;
    default: return cudaErrorInvalidValue;
    }
#undef VR_CYCLE
    return e;
}

}  // namespace vr
