// vr_grad.cu -- adjoint kernels of the frame: gradients of a loss on the image
// with respect to the transfer-function table and the voxel values.
//
// The paper renders only forward; its sort-last pipeline (Sec. 2.2 per-rank
// rendering, Sec. 3/4 compositing) is differentiated here step by step with the
// chain rule:
//   composite: I = C_front + F_b (C_b + (1 - A_b) R_b), with F_b the
//     transmittance in front of brick b and (R_b, 1 - Tb_b) the composite of the
//     bricks behind it: dI_rgb/dC_b = F_b, dI_rgb/dA_b = -F_b R_b,
//     dI_A/dA_b = F_b Tb_b;
//   per brick (C_{k+1} = C_k + T_k a_k c_k, T_{k+1} = T_k (1 - a_k), A = 1 - T_n),
//     back to front with lambda_T(n) = -dL/dA and lambda_C = dL/dC:
//     dL/dc_k = lambda_C T_k a_k, dL/da_k = T_k (lambda_C . c_k - lambda_T(k+1)),
//     lambda_T(k) = lambda_T(k+1) (1 - a_k) + a_k (lambda_C . c_k);
//   table lerp and trilinear weights as in the forward pass.
// T_k is never obtained by dividing by (1 - a): the march adjoint keeps the
// transmittance at every S-th sample of the forward pass (checkpoints) and
// recomputes each segment forward before walking it backwards.
#include "vr_device.cuh"

namespace vr {
namespace {

using dev::Quad;

// Composite adjoint: per pixel, the front transmittance of each brick (forward
// sweep) and the composite behind it (backward sweep) give the gradient of the
// brick's partial (dL/dC rgb, dL/dA), written in the partial pool's layout.
__global__ void __launch_bounds__(256) composite_grad_kernel(const __grid_constant__ CompositeGradParams p)
{
    __shared__ int s_brick[kMaxBricks];
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
            if (ov) s_brick[m + __popc(bal & ((1u << tid) - 1u))] = b;
            m += __popc(bal);
        }
        if (tid == 0) s_m = m;
    }
    __syncthreads();
    const int m = s_m;
    const int px = tx0 + threadIdx.x, py = ty0 + threadIdx.y;
    if (px >= p.W || py >= p.H) return;
    const float4 g = p.grad_img[static_cast<long long>(py) * p.W + px];
    auto at = [&](int b) {
        const int x0 = p.rect[b][0], y0 = p.rect[b][1], w = p.rect[b][2], h = p.rect[b][3];
        return (px >= x0 && px < x0 + w && py >= y0 && py < y0 + h)
                   ? p.poff[b] + static_cast<long long>(py - y0) * w + (px - x0)
                   : -1LL;
    };
    float F[kMaxBricks];  // transmittance in front of listed brick i
    float front = 1.0f;
    for (int i = 0; i < m; ++i) {
        F[i] = front;
        const long long o = at(s_brick[i]);
        if (o >= 0) front *= 1.0f - p.partials[o].w;
    }
    float R0 = 0.f, R1 = 0.f, R2 = 0.f, Tb = 1.0f;
    for (int i = m - 1; i >= 0; --i) {
        const long long o = at(s_brick[i]);
        if (o < 0) continue;
        const float4 P = p.partials[o];
        const float f = F[i];
        const float gA = f * (g.w * Tb - (g.x * R0 + g.y * R1 + g.z * R2));
        p.grad_partials[o] = make_float4(f * g.x, f * g.y, f * g.z, gA);
        const float keep = 1.0f - P.w;
        R0 = fmaf(keep, R0, P.x);
        R1 = fmaf(keep, R1, P.y);
        R2 = fmaf(keep, R2, P.z);
        Tb *= keep;
    }
}

// March adjoint: one thread per pixel of a brick's footprint (the forward
// decomposition). Per thread: forward over the owned run keeping T at every
// S-th sample, then segments back to front (forward recompute storing T_k,
// then the per-sample adjoint). Table gradients gather in shared memory per
// block; voxel gradients go to global memory with atomics on the global voxel
// index (halo copies alias their neighbours' voxels), once per run of samples
// in one cell.
template <typename S>
__global__ void __launch_bounds__(128) march_grad_kernel(const __grid_constant__ MarchParams p, GradArgs ga)
{
    constexpr int kMaxSeg = 64;  // checkpoints and segment length: runs up to 4096 samples
    extern __shared__ float s_gtf[];
    for (int i = threadIdx.x; i < 4 * p.ntf; i += blockDim.x) s_gtf[i] = 0.0f;
    __syncthreads();

    const int item = blockIdx.x;
    const BrickLaunch &B = p.b[dev::find_brick(p, item)];
    const int local = item - B.item_begin;
    const int ty = local / B.tiles_x, tx = local - ty * B.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rx = tx * p.tile_w + (warp & 1) * p.pw + (lane & (p.pw - 1));
    const int ry = ty * p.tile_h + (warp >> 1) * (32 / p.pw) + lane / p.pw;
    float4 gp = make_float4(0.f, 0.f, 0.f, 0.f);
    if (rx < B.rect[2] && ry < B.rect[3]) gp = ga.grad_partials[B.poff + static_cast<long long>(ry) * B.rect[2] + rx];
    dev::OwnedRun run;
    run.ka = 0;
    run.kb = -1;
    if (gp.x != 0.f || gp.y != 0.f || gp.z != 0.f || gp.w != 0.f)
        dev::owned_run(p, B, B.rect[0] + rx, B.rect[1] + ry, run);
    const int n = run.kb - run.ka + 1;
    int seg = max(16, (n + kMaxSeg - 1) / kMaxSeg);
    if (n > kMaxSeg * kMaxSeg) {
        atomicOr(ga.error, 1);  // run longer than the checkpoint storage: skipped, reported
        run.kb = run.ka - 1;
    }
    if (run.ka <= run.kb) {
        using Q = typename Quad<S>::type;
        const Q *vox = static_cast<const Q *>(p.data) + B.base;
        const int nbx = B.sx / 2, nby = B.sy / 2;
        const int imax = B.hi[0] - B.lo[0], jmax = B.hi[1] - B.lo[1], kmax = B.hi[2] - B.lo[2];
        const float xmax = static_cast<float>(p.ntf - 1);
        // one sample: cell, weights, scalar, table coordinate and entry
        struct Smp {
            int i, j, k, ti;
            float wx, wy, wz, x, w;
            float4 e0, de;
        };
        auto eval = [&](int kk, Smp &q) {
            const float h = static_cast<float>(kk) + 0.5f;
            const float vx = fmaf(h, run.step[0], run.base[0]);
            const float vy = fmaf(h, run.step[1], run.base[1]);
            const float vz = fmaf(h, run.step[2], run.base[2]);
            const float flx = floorf(vx), fly = floorf(vy), flz = floorf(vz);
            q.wx = vx - flx;
            q.wy = vy - fly;
            q.wz = vz - flz;
            q.i = min(max(static_cast<int>(flx), 0), imax);
            q.j = min(max(static_cast<int>(fly), 0), jmax);
            q.k = min(max(static_cast<int>(flz), 0), kmax);
            float4 a0, a1;
            if constexpr (Quad<S>::octet) {
                Quad<S>::load2(vox + quad_index(q.i, q.j, q.k, nbx, nby), a0, a1);
            } else {
                a0 = Quad<S>::load(vox + quad_index(q.i, q.j, q.k, nbx, nby));
                a1 = Quad<S>::load(vox + quad_index(q.i, q.j, q.k + 1, nbx, nby));
            }
            const float c00 = fmaf(q.wx, a0.y - a0.x, a0.x), c10 = fmaf(q.wx, a0.w - a0.z, a0.z);
            const float c01 = fmaf(q.wx, a1.y - a1.x, a1.x), c11 = fmaf(q.wx, a1.w - a1.z, a1.z);
            const float c0 = fmaf(q.wy, c10 - c00, c00), c1 = fmaf(q.wy, c11 - c01, c01);
            const float s = fmaf(q.wz, c1 - c0, c0);
            q.x = fmaf(s, p.tf_scale, p.tf_bias);
            const float x = fminf(fmaxf(q.x, 0.0f), xmax);
            q.ti = static_cast<int>(x);
            q.w = x - static_cast<float>(q.ti);
            q.e0 = __ldg(p.tf + 2 * q.ti);
            q.de = __ldg(p.tf + 2 * q.ti + 1);
        };
        float ck[kMaxSeg];  // T at the start of each segment
        float T = 1.0f;
        for (int kk = run.ka; kk <= run.kb; ++kk) {
            const int r = kk - run.ka;
            if (r % seg == 0) ck[r / seg] = T;
            Smp q;
            eval(kk, q);
            T = T - T * fmaf(q.w, q.de.w, q.e0.w);
        }
        const int nseg = (n + seg - 1) / seg;
        float lamT = -gp.w;
        float Ts[kMaxSeg];
        // voxel gradients of consecutive samples in one cell are summed in
        // registers and added to global memory once per cell (8 atomics)
        int cur_i = -1, cur_j = 0, cur_k = 0;
        float acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = 0.0f;
        // likewise table gradients of consecutive samples in one table interval
        // (entries ti and ti + 1) are summed before the shared-memory atomics
        int cur_ti = -1;
        float at0[4], at1[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) at0[c] = at1[c] = 0.0f;
        auto flush_tf = [&]() {
            if (cur_ti < 0) return;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                atomicAdd(&s_gtf[4 * cur_ti + c], at0[c]);
                if (cur_ti + 1 < p.ntf && at1[c] != 0.0f) atomicAdd(&s_gtf[4 * (cur_ti + 1) + c], at1[c]);
            }
        };
        auto flush = [&]() {
            if (cur_i < 0) return;
            const int gx0 = min(max(B.lo[0] - 1 + cur_i, 0), ga.N[0] - 1), gx1 = min(max(B.lo[0] + cur_i, 0), ga.N[0] - 1);
            const int gy0 = min(max(B.lo[1] - 1 + cur_j, 0), ga.N[1] - 1), gy1 = min(max(B.lo[1] + cur_j, 0), ga.N[1] - 1);
            const int gz0 = min(max(B.lo[2] - 1 + cur_k, 0), ga.N[2] - 1), gz1 = min(max(B.lo[2] + cur_k, 0), ga.N[2] - 1);
            const long long nx = ga.N[0], nxy = static_cast<long long>(ga.N[0]) * ga.N[1];
            float *gv = ga.grad_vol;
            atomicAdd(gv + gz0 * nxy + gy0 * nx + gx0, acc[0]);
            atomicAdd(gv + gz0 * nxy + gy0 * nx + gx1, acc[1]);
            atomicAdd(gv + gz0 * nxy + gy1 * nx + gx0, acc[2]);
            atomicAdd(gv + gz0 * nxy + gy1 * nx + gx1, acc[3]);
            atomicAdd(gv + gz1 * nxy + gy0 * nx + gx0, acc[4]);
            atomicAdd(gv + gz1 * nxy + gy0 * nx + gx1, acc[5]);
            atomicAdd(gv + gz1 * nxy + gy1 * nx + gx0, acc[6]);
            atomicAdd(gv + gz1 * nxy + gy1 * nx + gx1, acc[7]);
        };
        for (int sg = nseg - 1; sg >= 0; --sg) {
            const int k0 = run.ka + sg * seg, k1 = min(run.kb, k0 + seg - 1);
            float t = ck[sg];
            for (int kk = k0; kk <= k1; ++kk) {
                Ts[kk - k0] = t;
                Smp q;
                eval(kk, q);
                t = t - t * fmaf(q.w, q.de.w, q.e0.w);
            }
            for (int kk = k1; kk >= k0; --kk) {
                Smp q;
                eval(kk, q);
                const float Tk = Ts[kk - k0];
                const float r = fmaf(q.w, q.de.x, q.e0.x), g = fmaf(q.w, q.de.y, q.e0.y);
                const float b = fmaf(q.w, q.de.z, q.e0.z), a = fmaf(q.w, q.de.w, q.e0.w);
                const float gdotc = gp.x * r + gp.y * g + gp.z * b;
                const float ta = Tk * a;
                const float g4[4] = {gp.x * ta, gp.y * ta, gp.z * ta, Tk * (gdotc - lamT)};
                lamT = lamT * (1.0f - a) + a * gdotc;
                // table: rgba = (1-w) T[i] + w T[i+1]
                const float w0 = 1.0f - q.w;
                if (q.ti != cur_ti) {
                    flush_tf();
                    cur_ti = q.ti;
#pragma unroll
                    for (int c = 0; c < 4; ++c) at0[c] = at1[c] = 0.0f;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    at0[c] = fmaf(w0, g4[c], at0[c]);
                    at1[c] = fmaf(q.w, g4[c], at1[c]);
                }
                // scalar: ds = (g . (T[i+1] - T[i])) dx/ds where the table coordinate is not clamped
                if (ga.grad_vol && q.x > 0.0f && q.x < xmax) {
                    const float ds = (g4[0] * q.de.x + g4[1] * q.de.y + g4[2] * q.de.z + g4[3] * q.de.w) * p.tf_scale;
                    if (q.i != cur_i || q.j != cur_j || q.k != cur_k) {
                        flush();
                        cur_i = q.i;
                        cur_j = q.j;
                        cur_k = q.k;
#pragma unroll
                        for (int c = 0; c < 8; ++c) acc[c] = 0.0f;
                    }
                    const float ux = 1.0f - q.wx, uy = 1.0f - q.wy, uz = 1.0f - q.wz;
                    const float dz0 = ds * uz, dz1 = ds * q.wz;
                    acc[0] = fmaf(dz0, ux * uy, acc[0]);
                    acc[1] = fmaf(dz0, q.wx * uy, acc[1]);
                    acc[2] = fmaf(dz0, ux * q.wy, acc[2]);
                    acc[3] = fmaf(dz0, q.wx * q.wy, acc[3]);
                    acc[4] = fmaf(dz1, ux * uy, acc[4]);
                    acc[5] = fmaf(dz1, q.wx * uy, acc[5]);
                    acc[6] = fmaf(dz1, ux * q.wy, acc[6]);
                    acc[7] = fmaf(dz1, q.wx * q.wy, acc[7]);
                }
            }
        }
        if (ga.grad_vol) flush();
        flush_tf();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * p.ntf; i += blockDim.x)
        if (s_gtf[i] != 0.0f) atomicAdd(ga.grad_tf + i, s_gtf[i]);
}

}  // namespace

cudaError_t launch_composite_grad(const CompositeGradParams &p, cudaStream_t s)
{
    if (p.W <= 0 || p.H <= 0) return cudaSuccess;
    dim3 block(kCompW, kCompH);
    dim3 grid((p.W + kCompW - 1) / kCompW, (p.H + kCompH - 1) / kCompH);
    composite_grad_kernel<<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_march_grad(const MarchParams &p, const GradArgs &g, int kind, cudaStream_t s)
{
    if (p.n_items <= 0) return cudaSuccess;
    const size_t smem = 4 * static_cast<size_t>(p.ntf) * sizeof(float);
    switch (kind) {
    case kStoreF32: march_grad_kernel<float><<<p.n_items, 128, smem, s>>>(p, g); break;
    case kStoreBF16: march_grad_kernel<__nv_bfloat16><<<p.n_items, 128, smem, s>>>(p, g); break;
    case kStoreF16: march_grad_kernel<__half><<<p.n_items, 128, smem, s>>>(p, g); break;
    case kStoreBF16Oct: march_grad_kernel<dev::Octet<__nv_bfloat16>><<<p.n_items, 128, smem, s>>>(p, g); break;
    case kStoreF16Oct: march_grad_kernel<dev::Octet<__half>><<<p.n_items, 128, smem, s>>>(p, g); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace vr
