// vr_objects.h -- host-side objects of libvr (context, volume, frame) and the
// host helpers shared by vr_host.cpp and vr_batch.cu. Not part of the public ABI.
#pragma once

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "vr_internal.h"

namespace vr {
namespace host {

// Fault injection for tests (vr_debug_inject_fault): a one-shot plan that makes
// the device allocation or kernel launch after `after` successful ones fail on
// the host, without calling CUDA.
bool fault_now(int kind);  // kind: VR_FAULT_ALLOC or VR_FAULT_LAUNCH

template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes)
{
    if (fault_now(VR_FAULT_ALLOC)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}

// Named NVTX range around a public call (visible in timeline profilers; a no-op
// unless a tool is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

struct KdNode {
    int axis = -1;  // -1: leaf
    int cut = 0;    // voxel plane
    int child[2] = {-1, -1};
    int brick = -1;
};

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace host
}  // namespace vr

struct vr_frame_s {
    vr_ctx ctx = nullptr;
    int nb = 0;
    int W = 0, H = 0;
    std::vector<int> rects;        // nb x 4
    std::vector<int> order;        // nb
    std::vector<long long> poff;   // nb, float4 units
    long long total_px = 0;        // partial pixels (float4), 128-byte aligned per brick
    int tiles_x = 0, tiles_y = 0;  // composite tiles (kCompW x kCompTileH)
    long long pool_px = 0;         // float4 units of the pool: partials, then one mask per tile
    bool masks_ready = false;      // the masks were written by this frame's march
    float4 *d_part = nullptr;
    long long cap_px = 0;
    bool owned_by_ctx = false;
};

struct vr_ctx_s {
    int device = 0;
    std::string last_error;
    float4 *d_tf = nullptr;
    int ntf = 0;
    int tf_cap = 0;
    float vmin = 0.f, vmax = 1.f;
    bool has_tf = false;
    vr_camera cam{};
    bool has_cam = false;
    float step = 0.5f;
    float ert_alpha = 1.0f;
    std::vector<int> factors;
    int mode = 0;                  // 0: sort-last partials + composite; 1: ray-state cycling
    float opc_ref = 0.0f;          // opacity-correction reference step in voxels (0: off)
    int packet_width = 4;          // ray packet of the march: pw x (32/pw) pixels per warp
    bool staging = false;          // march float32 volumes with brick slabs staged in shared memory
    int cell_layout = 0;           // 16-bit volumes created next: 0 xy-quads, 1 octets (vr_set_cell_layout)
    unsigned long long *d_counter = nullptr;
    int *d_error = nullptr;        // device error word (vr_sync reports and clears it)
    bool count_samples = false;
    float4 *d_gpart = nullptr;     // partial gradients (backward), partial-pool layout
    long long gpart_cap = 0;
    vr_frame_s frame;              // context-owned frame for vr_render_frame
    // Pipelined frames (vr_set_frame_pipelining): vr_render_frame into device
    // memory alternates between `frame` and `frame2`, and its march may start
    // in the previous frame's composite when nothing the march reads before its
    // waits (bricks, table) has been written since that composite was launched
    // on the same stream: input_seq counts brick packs and table uploads.
    bool pipelining = true;
    vr_frame_s frame2;
    int sms = 0;                   // multiprocessors of the device (persistent composite grid)
    unsigned long long input_seq = 0;
    bool pipe_ready = false;
    cudaStream_t pipe_stream = nullptr;
    unsigned long long pipe_seq = 0;
    // per pool (frame, frame2): the last pipelined frame whose composite read it
    // and is done, and that composite's count of finished blocks (device);
    // pipelined frames are numbered from 1 and frame n uses pool n % 2
    unsigned long long *d_pool_done = nullptr;
    unsigned int *d_pool_count = nullptr;
    unsigned long long pool_frame = 0;
    float4 *d_img = nullptr;       // staging for host outputs
    long long img_cap = 0;
    // asynchronous host output: two staging images, copies on their own stream
    bool host_async = false;
    float4 *d_img2[2] = {nullptr, nullptr};
    long long img2_cap = 0;
    int img_next = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_rendered[2] = {nullptr, nullptr};
    cudaEvent_t ev_copied[2] = {nullptr, nullptr};
    int live_objects = 0;
    // kernel timing (vr_set_kernel_timing)
    bool timing = false;
    struct Timed {
        cudaEvent_t a, b;
        int kind;  // 0 march, 1 composite
    };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> event_pool;
};

struct vr_volume_s {
    vr_ctx ctx = nullptr;
    int dims[3] = {0, 0, 0};
    vr_dtype dtype = VR_F32;
    std::vector<int> boxes;        // nb x 6
    std::vector<long long> base;   // element offsets
    std::vector<vr::host::KdNode> tree;  // node 0 = root
    void *d_data = nullptr;
    long long bytes = 0;
    float *d_staging = nullptr;    // float32 source for asynchronous re-packs from host memory
    // scalar copy of the bricks for the staged march (float32 volumes created
    // while the context's staging was on): per brick, haloed voxels with rows
    // padded to sxp elements, starting at element sbase
    float *d_scalar = nullptr;
    std::vector<long long> sbase;
    std::vector<int> sxp;
    // a rank's share (vr_volume_create_share): held[b] != 0 for the bricks this
    // volume stores; empty = every brick. Bricks not held have no storage and
    // render as empty partials (the identity of "over").
    std::vector<char> held;
    bool holds(int b) const { return held.empty() || held[b]; }
    bool octets = false;           // 16-bit storage with both planes of a cell per element
    int kind() const { return vr::storage_kind(dtype, octets); }
};

namespace vr {
namespace host {

size_t elem_size(vr_dtype t);
size_t quad_size(vr_dtype t, bool octets = false);
long long brick_quads(const int *bx);
vr_status fail(vr_ctx ctx, vr_status s, const std::string &msg);
vr_status cuda_fail(vr_ctx ctx, cudaError_t e, const char *what);
int nmax3(const int d[3]);
void visibility_order(const std::vector<KdNode> &tree, int node, const vr_camera &cam, double nmax,
                      std::vector<int> &out);
struct Basis {
    double f[3], r[3], u[3];
    double tanx, tany;
};
bool make_basis(const vr_camera &c, Basis &B);
void footprint(const vr_camera &c, const Basis &B, const int box[6], double nmax, int rect[4]);
bool partition_plan(const int dims[3], const vr_partition *part, std::vector<int> &boxes,
                    std::vector<KdNode> &tree, const char **why);
// Per-view setup of a partitioned object (visibility order, footprints, launch
// table); reads only the geometry fields of `vol` (dims, boxes, tree, base, d_data).
vr_status prepare_frame(vr_ctx ctx, vr_volume vol, vr_frame_s &fr, MarchParams &mp);
vr_status ensure_frame(vr_ctx ctx, vr_frame_s &fr, long long px);
vr_status composite_to(vr_ctx ctx, vr_frame_s &fr, float *out, int out_on_device, cudaStream_t s);
// pipelined frames (vr_set_frame_pipelining; vr_host.cpp): the pool wait of
// a frame's march and the release by its composite
struct PoolSync {
    unsigned long long *done;
    unsigned int *count;
    unsigned long long frame;
    int pool;
};
bool pipelined_output(vr_ctx ctx, int out_on_device);
bool pipe_after(vr_ctx ctx, cudaStream_t s);
void pipe_launched(vr_ctx ctx, cudaStream_t s);
PoolSync pipe_frame(vr_ctx ctx);
vr_frame_s &pipe_pool(vr_ctx ctx, const PoolSync &sync);
vr_status composite_pipelined(vr_ctx ctx, vr_frame_s &fr, float *out, int out_on_device, cudaStream_t s,
                              const PoolSync &sync);
int timing_begin(vr_ctx ctx, int kind, cudaStream_t s);
void timing_end(vr_ctx ctx, int idx, cudaStream_t s);

}  // namespace host
}  // namespace vr

// Return the CUDA error of `call` as a vr_status with the context's message.
#define VR_CUDA(ctx, call)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// A kernel launch through a launcher, with the launch fault hook.
#define VR_LAUNCH(ctx, call)                                                              \
    do {                                                                                  \
        if (vr::host::fault_now(VR_FAULT_LAUNCH))                                          \
            return cuda_fail(ctx, cudaErrorLaunchFailure, #call " (injected fault)");     \
        VR_CUDA(ctx, call);                                                               \
    } while (0)
