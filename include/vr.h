/*
 * vr.h -- C ABI of libvr, a GB300 (sm_103a) data-parallel volume renderer.
 *
 * The library renders one scalar volume split into bricks that all live on
 * one GPU. Each brick stands in for one rank of the paper's cluster
 * (arXiv:2501.01628, Sec. 2.2: the data is spatially distributed across ranks,
 * each rank getting a share, possibly uneven; Sec. 4: several data parts are
 * recombined per GPU). A frame is rendered in two steps that follow the paper's
 * statement of the problem (Sec. 3: a collective render call retires pixels into
 * a framebuffer that ends up in one place; Sec. 4: processes "render and
 * composite images"):
 *   1. per-brick emission-absorption ray marching on a global sample lattice,
 *      giving one partial RGBA image per brick (vr_render_partials), and
 *   2. sort-last compositing of the partials with the "over" operator in
 *      front-to-back visibility order (vr_composite).
 * The paper gives no rendering formula; the library implements the standard
 * emission-absorption model (Max 1995) with these definitions:
 *   - world box [0,Nx/Nmax]x[0,Ny/Nmax]x[0,Nz/Nmax], voxel centres at (i+.5)/Nmax;
 *   - samples t_k = t_in + (k+1/2) dt, dt = step_voxels/Nmax, while t_k < t_out,
 *     [t_in,t_out) the ray's interval in the whole-volume box (t_in >= 0);
 *   - sample k belongs to the brick whose voxel box holds the cell
 *     clamp(floor(p*Nmax), 0, N-1) of its position p;
 *   - trilinear reconstruction with clamp-to-edge; 1D RGBA table lookup with
 *     linear interpolation over [vmin, vmax]; per-sample opacity = table alpha;
 *   - per brick: C += T*alpha*rgb, T *= (1-alpha) from C=0, T=1; the partial is
 *     (C, 1-T) (premultiplied colour); optional early termination per brick
 *     when T <= 1 - ert_alpha;
 *   - composite: C <- C + (1-A) C_b, A <- A + (1-A) A_b, bricks front to back.
 *
 * Conventions for every call:
 *   - Return value: VR_OK or an error code; no call aborts or exits. The text
 *     of the last error of a context is available from vr_last_error().
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Device work is asynchronous on that stream unless stated.
 *   - Pointers named *_dev are device pointers owned by the caller; the
 *     library never frees them. Objects created by vr_*_create / vr_render_*
 *     are owned by the library until the matching release call.
 *   - A context is not thread-safe; use one context per host thread.
 *   - Images are row-major [height][width][4] float32 RGBA, row 0 at the
 *     bottom of the view (pixel (px,py) has its centre at ((px+.5)/W, (py+.5)/H)
 *     of the image plane).
 */
#ifndef VR_H
#define VR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vr_ctx_s *vr_ctx;
typedef struct vr_volume_s *vr_volume;
typedef struct vr_frame_s *vr_frame;
typedef struct vr_batch_s *vr_batch;
typedef struct vr_mesh_s *vr_mesh;

typedef enum {
    VR_OK = 0,
    VR_ERR_ARG = 1,     /* invalid argument (bad dims, partition that does not tile, ...) */
    VR_ERR_OOM = 2,     /* device or host allocation failed */
    VR_ERR_CUDA = 3,    /* a CUDA runtime call failed; see vr_last_error */
    VR_ERR_STATE = 4,   /* call out of order (no camera / transfer function yet, ...) */
    VR_ERR_TIMEOUT = 5, /* a bounded device-side wait gave up */
    VR_ERR_BOUNDS = 6   /* a device-side index check failed */
} vr_status;

typedef enum { VR_F32 = 0, VR_BF16 = 1, VR_F16 = 2 } vr_dtype;

typedef enum { VR_PART_GRID = 0, VR_PART_KD = 1, VR_PART_BOXES = 2 } vr_partition_kind;

/* Camera (Sec. 2.1: primary rays start at the virtual camera).
 * Basis f = dir/|dir|, r = normalise(up x f), u = f x r.
 * Orthographic (ortho != 0): ray origin eye + ((px+.5)/W-.5) ortho_w r
 *   + ((py+.5)/H-.5) ortho_h u, direction f.
 * Perspective: origin eye, direction normalise(f + sx r + sy u) with
 *   sy = ((py+.5)/H*2-1) tan(fovy/2), sx = ((px+.5)/W*2-1) tan(fovy/2) W/H. */
typedef struct {
    int ortho;
    double eye[3], dir[3], up[3];
    double fovy_deg, ortho_w, ortho_h;
    int width, height;
} vr_camera;

/* Brick partition of the volume (Sec. 2.2 spatial distribution; Sec. 4 uneven
 * shares and several parts per GPU).
 *   VR_PART_GRID : grid[0] x grid[1] x grid[2] bricks, boundaries floor(N j/g),
 *                  brick id (bz*gy + by)*gx + bx.
 *   VR_PART_KD   : n_bricks leaves; repeatedly the leaf with the most voxels
 *                  (ties: lowest id) is cut across its longest axis (ties:
 *                  x, y, z) at lo + round(cut_fracs[j]*extent), clamped so both
 *                  halves are non-empty; the low half keeps the id, the high
 *                  half gets the next id. cut_fracs holds n_bricks-1 values.
 *   VR_PART_BOXES: n_bricks half-open voxel boxes (lo x,y,z, hi x,y,z) that
 *                  tile the volume and can be separated by axis-aligned cuts
 *                  (needed for a visibility order); otherwise VR_ERR_ARG.
 * At most VR_MAX_BRICKS bricks. vr_volume_create also refuses (VR_ERR_ARG) a brick
 * whose haloed storage exceeds 2^31 - 1 xy-quads (about 1290^3 voxels). */
#define VR_MAX_BRICKS 128
typedef struct {
    int kind;
    int grid[3];
    int n_bricks;
    const double *cut_fracs;
    const int *boxes;
} vr_partition;

/* ---- host-only planning (no GPU needed) -------------------------------- */

/* Bricks that `part` produces for a dims[0] x dims[1] x dims[2] volume: their
 * count and, if `boxes` is not NULL, their voxel boxes (n x 6 ints). Fails with
 * VR_ERR_ARG for an invalid description or boxes that do not tile the volume
 * with axis-aligned cuts. */
vr_status vr_partition_boxes(const int dims[3], const vr_partition *part, int *n_bricks, int *boxes);
/* Per-view plan of a partitioned volume: front-to-back brick order (n ids,
 * from a traversal of the partition's kd tree towards the eye, or along the view
 * direction for orthographic cameras; ties resolved low side first) and the
 * conservative screen rectangle of each brick (n x 4: x0, y0, w, h; w = h = 0
 * when the brick cannot be seen). Either output may be NULL. */
vr_status vr_plan_view(const int dims[3], const vr_partition *part, const vr_camera *cam, int *order,
                       int *rects);

/* ---- context ----------------------------------------------------------- */

/* Create a context on CUDA device `cuda_device`. */
vr_status vr_create(int cuda_device, vr_ctx *out);
/* Destroy a context; its volumes and frames must have been released. Waits for
 * the device. */
vr_status vr_destroy(vr_ctx ctx);
const char *vr_status_string(vr_status s);
/* Text of the last error of `ctx` ("" if none); valid until the next call. */
const char *vr_last_error(vr_ctx ctx);
/* Wait for `stream` and report any device-side error word set by a kernel
 * (VR_ERR_TIMEOUT for a bounded wait that gave up, VR_ERR_BOUNDS for an
 * adjoint run beyond its checkpoint storage), clearing it. */
vr_status vr_sync(vr_ctx ctx, void *stream);

/* ---- volume (the distributed World of Sec. 3, all bricks on this GPU) ---- */

/* Create a volume of dims[0] x dims[1] x dims[2] voxels (x fastest) from the
 * float32 array `src` (host memory if src_on_device == 0, else device memory;
 * not retained) and pack it into brick-major storage of type `storage`
 * (float32, or bfloat16 / float16 rounded to nearest even) with a one-voxel
 * halo per brick holding the neighbouring (edge-clamped) voxels. The packing
 * runs on `stream` and is complete when this call returns. */
vr_status vr_volume_create(vr_ctx ctx, const int dims[3], vr_dtype storage,
                           const vr_partition *part, const float *src, int src_on_device,
                           void *stream, vr_volume *out);
/* A rank's share of a volume (Sec. 2.2: the data is spatially distributed,
 * each rank holding a share; Sec. 4: shares may be uneven): as
 * vr_volume_create, but only the n_held bricks listed in `held` (distinct
 * brick ids of `part`) are stored, packed and marched. Bricks not held render
 * as empty partials -- the identity of "over" -- so vr_render_frame gives this
 * rank's image: its bricks composited front to back. `src` is still the whole
 * volume (only the held bricks and their halos are read). Shares cannot be
 * batched (vr_batch_create returns VR_ERR_ARG). */
vr_status vr_volume_create_share(vr_ctx ctx, const int dims[3], vr_dtype storage, const vr_partition *part,
                                 int n_held, const int *held, const float *src, int src_on_device, void *stream,
                                 vr_volume *out);
vr_status vr_volume_release(vr_volume vol);
/* Number of bricks, their voxel boxes (n x 6 ints, may be NULL) and the bytes
 * of brick storage in device memory (may be NULL). */
vr_status vr_volume_info(vr_volume vol, int *n_bricks, int *boxes, long long *storage_bytes);
/* Copy brick `brick`'s haloed storage, (bx+2)(by+2)(bz+2) elements x fastest,
 * into host memory `dst` of `bytes` bytes (synchronous). For tests. */
vr_status vr_volume_read_brick(vr_volume vol, int brick, void *dst, size_t bytes);

/* ---- renderer state --------------------------------------------------- */

/* Transfer function: 2 <= n <= 1024 RGBA entries (entry i at u = i/(n-1)), scalar range
 * [vmin, vmax] with vmax > vmin. `rgba` is host memory (on_device == 0) or
 * device memory; it is copied, synchronously. */
vr_status vr_set_transfer_function(vr_ctx ctx, const float *rgba, int n, float vmin, float vmax,
                                   int on_device);
vr_status vr_set_camera(vr_ctx ctx, const vr_camera *cam);
/* step_voxels > 0 (default 0.5); ert_alpha in (0,1) enables early ray
 * termination per brick, >= 1 disables it (default 1). */
vr_status vr_set_render_params(vr_ctx ctx, float step_voxels, float ert_alpha);
/* Compositing association tree: n_factors factors whose product equals the
 * brick count (radix-k rounds: groups of factors[0] consecutive partials in
 * visibility order are combined first, then groups of factors[1] of those, ...).
 * n_factors == 0 selects direct k-way compositing. At most 8 factors. */
vr_status vr_set_composite_schedule(vr_ctx ctx, int n_factors, const int *factors);
/* Opacity correction (off by default): with ref_step_voxels > 0, each sample's
 * table opacity alpha is replaced by 1 - (1 - alpha)^(step_voxels /
 * ref_step_voxels), so the table means "opacity per ref_step_voxels of path" and
 * the image no longer depends on the step (the paper fixes no optical model;
 * this is the standard correction of emission-absorption ray casting).
 * ref_step_voxels == 0 turns it off. Not available in vr_render_backward. */
vr_status vr_set_opacity_correction(vr_ctx ctx, float ref_step_voxels);
/* Host outputs (out_on_device == 0 in vr_composite / vr_render_frame) are
 * synchronous by default: the call returns with the image in host memory. With
 * on != 0 the call returns without waiting for its own image; the image is
 * copied from one of two device staging buffers on the context's own copy
 * stream, overlapping the next frame's rendering, and is in host memory after
 * vr_sync(ctx, stream). A call first waits on the host until the staging
 * buffer's previous copy (two calls back) is done (inside stream capture the
 * stream waits instead). Use pinned host buffers, and a different host buffer
 * for each of two consecutive frames. */
vr_status vr_set_host_output_async(vr_ctx ctx, int on);
/* Ray-packet shape of the march: each warp marches packet_width x
 * (32/packet_width) neighbouring pixels (4, 8 or 16; default 4). The image does
 * not depend on it; the speed does (it sets how compactly a warp's rays touch
 * the brick's cache lines). */
vr_status vr_set_packet_width(vr_ctx ctx, int packet_width);
/* March variant for float32 volumes (off by default). With on != 0, volumes
 * created afterwards also keep a scalar copy of their bricks (one float per
 * haloed voxel, about a quarter of the xy-quad storage), and the march of
 * those volumes stages the brick voxels of each 8x16-pixel tile in shared
 * memory, slab by slab in depth (bulk asynchronous copies, cp.async.bulk,
 * completing on an mbarrier, two stages per block), instead of reading
 * xy-quads through L1. The image is the same bit for bit; the speed differs
 * (brick tiles staged for ray packets; on the 1080p orbit workload it is
 * slower than the xy-quad march). Volumes without the scalar copy (other
 * storage types, or created while staging was off) keep the xy-quad march.
 * Each bounded wait for a staged slab that gives up makes the next vr_sync
 * return VR_ERR_TIMEOUT. */
vr_status vr_set_march_staging(vr_ctx ctx, int on);
/* Pipelined frames (on by default). With on != 0, vr_render_frame calls into
 * device memory, or into host memory with asynchronous host output
 * (vr_set_host_output_async), alternate between two context-owned frames
 * (partial pools), and the composite runs as a persistent grid of two blocks
 * per multiprocessor that signals at its start, so the next such call's march
 * can start while this frame's march drains and its composite runs
 * (programmatic dependent launch; Sec. 3's render-then-composite per frame,
 * overlapped between consecutive frames). Ordering stays that of the stream:
 * the overlapping march's tile masks wait for the previous composite to
 * complete (so the march completes only after it), its partials wait only for
 * the composite that last read their pool (two frames back; a bounded wait on
 * a device flag that composite releases -- if it gives up, the next vr_sync
 * returns VR_ERR_TIMEOUT and the frame's partials are not written), and the
 * march overlaps only when the previous pipelined frame was launched on the
 * same stream and no brick pack (volume create or update) and no
 * transfer-function upload of this context
 * came in between. Images are bit-identical either way. Kernel timing,
 * synchronous host outputs and the staged march use the plain sequence (one
 * frame, one block per composite tile). Costs a second partial pool per
 * context. Mesh frames (vr_render_mesh_frame) are pipelined the same way;
 * ray-state cycling frames (vr_set_render_mode 1) too, their kernel writing
 * its image after the previous frame's last kernel completes. */
vr_status vr_set_frame_pipelining(vr_ctx ctx, int on);
/* Test hook of the pipelined frames' bounded pool wait: advances the context's
 * frame count by two without rendering, so the next pipelined frame's march
 * waits for a pool release that never comes; after its bounded wait (2^20
 * polls per thread) it skips its partials, and the next vr_sync returns
 * VR_ERR_TIMEOUT and re-arms the pool flags, so the following frames render
 * normally. Nothing faults or hangs. */
vr_status vr_debug_pipeline_gap(vr_ctx ctx);
/* Cell layout of bfloat16 / float16 volumes created afterwards (the precision
 * form: 16-bit storage, float32 arithmetic). 0 (default): xy-quads, four
 * voxels of one plane per 8-byte element, two loads per sample. 1: octets,
 * both planes of a cell in one 16-byte element, one load per sample: twice the
 * memory of xy-quads (as much as float32 xy-quads), faster where the march is
 * bound by its loads. The image is the same bit for bit. Float32 volumes
 * always use xy-quads (float32 octets measured slower). Volumes of one batch
 * must share the layout. VR_ERR_ARG for another value. */
vr_status vr_set_cell_layout(vr_ctx ctx, int layout);
/* Frame algorithm of vr_render_frame.
 *   0 (default): sort-last -- one partial image per brick, then the "over"
 *     composite (the steps above).
 *   1: ray-state cycling -- each ray carries one (C, T) through the bricks in
 *     front-to-back order and writes its pixel directly (the paper's ray-queue
 *     cycling, where every ray visits every rank, Sec. 2.2 and 3, restated for
 *     bricks on one GPU). No partial images; early termination applies to the
 *     whole ray (T <= 1 - ert_alpha), not per brick. With early termination off
 *     it computes the same image as mode 0 up to rounding.
 * vr_render_partials, vr_composite and vr_render_backward always use the
 * sort-last steps. */
vr_status vr_set_render_mode(vr_ctx ctx, int mode);
/* When on, every march launch also counts executed samples (see
 * vr_get_sample_count). Off by default. The counting launches also check that
 * every executed sample's quads lie inside its brick's storage (the index clamps
 * of the march only guard memory); a violation makes the next vr_sync return
 * VR_ERR_BOUNDS. */
vr_status vr_set_count_samples(vr_ctx ctx, int on);
/* Samples counted since the last call (synchronises the context's device). */
vr_status vr_get_sample_count(vr_ctx ctx, long long *count);

/* When on, the library records a CUDA event pair on the launching stream
 * around each of its march and composite kernel launches. Off by default.
 * The events cost time (about 10 us per 1080p frame on a GB300) and keep the
 * composite from starting in the march's tail, so switch timing on for a
 * subset of frames when measuring throughput. */
vr_status vr_set_kernel_timing(vr_ctx ctx, int on);
/* Summed device time (ms) and launch count of the march and composite kernels
 * recorded since the last call (waits for the recorded events). Any output may
 * be NULL. */
vr_status vr_get_kernel_timing(vr_ctx ctx, double *march_ms, long long *march_launches,
                               double *composite_ms, long long *composite_launches);

/* ---- rendering --------------------------------------------------------- */

/* Step 1: march every brick, producing one partial RGBA32F image per brick
 * over the brick's screen footprint rectangle. The frame (partials, rectangles,
 * visibility order) belongs to the library until vr_frame_release. */
vr_status vr_render_partials(vr_ctx ctx, vr_volume vol, vr_frame *out, void *stream);
/* Frame layout: rects n x 4 (x0, y0, w, h) per brick id, order n brick ids front
 * to back (either may be NULL). */
vr_status vr_frame_info(vr_frame fr, int *n_bricks, int *rects, int *order);
/* Device pointer to brick `brick`'s partial: h rows of w float4 (RGBA). */
vr_status vr_frame_partial(vr_frame fr, int brick, const float **dev_ptr);
/* Step 2: composite the frame's partials front to back with the context's
 * schedule into out_rgba (device memory if out_on_device, else host memory; a
 * host output makes the call synchronous). */
vr_status vr_composite(vr_ctx ctx, vr_frame fr, float *out_rgba, int out_on_device, void *stream);
vr_status vr_frame_release(vr_frame fr);
/* Sec. 3: the ranks' images end up composited into one framebuffer. out_dev =
 * images_dev[0] over images_dev[1] over ... over images_dev[n-1], pixel by pixel
 * (front to back; premultiplied RGBA, "over" as above), for `pixels` pixels of
 * float32 RGBA in device memory (1 <= n <= VR_MAX_BRICKS; every pointer 16-byte
 * aligned, else VR_ERR_ARG). `images_dev` is a host array of device pointers.
 * out_dev may be images_dev[0]. This is the combining step of each round of a
 * radix-k image exchange between GPUs (paper_2501_01628_gb300/sharded.py). */
vr_status vr_composite_images(vr_ctx ctx, int n, const float *const *images_dev, float *out_dev, long long pixels,
                              void *stream);
/* Steps 1 + 2 with a context-owned frame (no allocation once warm). */
vr_status vr_render_frame(vr_ctx ctx, vr_volume vol, float *out_rgba, int out_on_device,
                          void *stream);

/* ---- batched form: many renders in one launch ------------------------------ */

/* A batch renders every (volume, view) pair -- render r = v * n_views + w --
 * into out_rgba_dev (n_volumes x n_views x H x W x 4 float32, device), e.g. the
 * time steps and fields of a time-varying data set (Sec. 4) seen from many
 * views (replication of resident data, Sec. 2.2). All renders and their
 * compositing run in ONE persistent, cooperative kernel, captured with its
 * counter resets in a CUDA graph; vr_batch_launch replays that graph.
 *   - volumes: same dims, partition and storage type; per-volume classification
 *     range vmins/vmaxs (NULL: the context's range); the context's transfer
 *     function table, step and early termination are captured at creation;
 *   - cameras: same image size; direct (non-radix) front-to-back composite;
 *   - work items (the (brick, tile) march items of render r, then its composite
 *     tiles) are claimed in order from one counter; partial images live in a
 *     ring of slots reused once composited; device-side waits are bounded and
 *     report VR_ERR_TIMEOUT through vr_sync instead of hanging.
 * The batch belongs to the library until vr_batch_release. */
vr_status vr_batch_create(vr_ctx ctx, int n_volumes, const vr_volume *vols, const float *vmins, const float *vmaxs,
                          int n_views, const vr_camera *cams, float *out_rgba_dev, vr_batch *out);
/* Launch the whole batch on `stream` (asynchronous). */
vr_status vr_batch_launch(vr_batch batch, void *stream);
/* Time the candidates -- work order (0: render by render; 1: volume by volume
 * with every view marching one brick before the next, so the brick stays in L2),
 * ray-packet shape (4x8, 8x4, 16x2 pixels per warp) and resident blocks per SM --
 * with one launch each (synchronous) and keep the fastest; with a non-NULL
 * cache_path the choice is read from / appended to a text cache keyed by device
 * name and batch shape. chosen (may be NULL, else 4 ints) gets {packet width,
 * blocks per SM, ring slots, work order}. */
vr_status vr_batch_autotune(vr_batch batch, void *stream, const char *cache_path, int *chosen);
/* Set the configuration directly: packet_width 4, 8 or 16; blocks_per_sm (0 =
 * as many as fit); order 0 or 1 as for vr_batch_autotune. */
vr_status vr_batch_configure(vr_batch batch, int packet_width, int blocks_per_sm, int order);
vr_status vr_batch_release(vr_batch batch);
/* Test hook for the bounded waits (the paper has no counterpart). Rebuilds the
 * batch's graph so that each device-side wait gives up after `wait_limit`
 * sleeps of about 128 ns (0 restores the default of 2^25, about 4 s) and the
 * composite tiles of unit 0 wait for `extra_march` more finished march items
 * than exist. With extra_march > 0 those waits cannot succeed: the first to give
 * up sets the device error word, every other wait and claim stops, the launch
 * ends with some renders incomplete, and the next vr_sync returns
 * VR_ERR_TIMEOUT. Nothing faults or hangs. (0, 0) restores normal operation.
 * VR_ERR_ARG for negative arguments. */
vr_status vr_batch_debug_wait(vr_batch batch, int wait_limit, int extra_march);

/* ---- differentiation ------------------------------------------------------ */

/* Replace the voxel values of `vol` (same dims and partition) from the float32
 * array `src` (host if src_on_device == 0, else device) and re-pack its bricks
 * in place, on `stream`; complete when the call returns. No allocation for a
 * device source. */
vr_status vr_volume_update(vr_volume vol, const float *src, int src_on_device, void *stream);
/* As vr_volume_update, but asynchronous on `stream`: for time-varying data
 * streamed through a fixed device budget (Sec. 4: time steps are loaded and
 * later evicted rather than all held in GPU memory), the next step is uploaded
 * and packed on one stream while another renders. A host source must be pinned
 * memory for the copy to overlap; it is staged in a device buffer of the
 * volume's float32 size, allocated by the first such call and kept until
 * vr_volume_release. Order renders after the update with events. */
vr_status vr_volume_update_async(vr_volume vol, const float *src, int src_on_device, void *stream);
/* Gradient of a loss on the frame that vr_render_frame would produce with the
 * context's current camera, transfer function and parameters (the paper renders
 * only forward; this is the chain rule through the readings stated at the top
 * of this header). Given dL/dI in `grad_rgba_dev` (H x W x 4 float32, device),
 * ADDS dL/d(table) to `grad_tf_dev` (n x 4 float32, device) and, unless it is
 * NULL, dL/d(voxel) to `grad_density_dev` (Nz x Ny x Nx float32, device, the
 * original volume's indexing: halo copies are summed into the voxels they copy).
 * Recomputes the forward pass per brick; transmittances come from checkpoints,
 * never from division. Requires early termination off (VR_ERR_ARG otherwise).
 * Runs of more than 4096 owned samples in one brick are skipped and reported as
 * VR_ERR_BOUNDS by vr_sync. Float atomics: results vary in the last bits
 * between runs. */
vr_status vr_render_backward(vr_ctx ctx, vr_volume vol, const float *grad_rgba_dev, float *grad_tf_dev,
                             float *grad_density_dev, void *stream);

/* ---- unstructured elements (tetrahedral meshes) ------------------------- */

/* Sec. 5: the paper renders a mixed finite-element data set kept in the
 * distribution its simulation used, each rank holding whole elements, unevenly
 * spread in space; Sec. 2.1: rays find the objects they meet through a bounding
 * volume hierarchy. Here the elements are tetrahedra (a mixed mesh enters as its
 * tetrahedral decomposition) and the ranks are the bricks of `part`.
 *
 * Create a mesh volume from HOST arrays (copied; the library owns the result
 * until vr_mesh_release):
 *   verts   n_verts x 3 float32 world positions inside [0, dims/Nmax];
 *   values  n_verts float32 vertex values;
 *   tets    n_tets x 4 int32 vertex indices (either orientation).
 * `dims` is the nominal lattice: as for a voxel volume it fixes the domain box,
 * the sample spacing (step_voxels / Nmax) and the sample ownership cells. Each
 * element belongs to the brick whose box holds its centroid's cell and must lie
 * inside that box (1e-3 voxel tolerance); each brick's elements must fill its box
 * without gaps or overlaps (volumes checked to 1e-4) and share faces only
 * pairwise. A violation, a degenerate element or an empty brick gives
 * VR_ERR_ARG. The per-brick BVHs and face adjacency are built on the host.
 *
 * Sampling (reading; the paper gives none): a lattice sample keeps the owner of
 * the voxel path (its cell's brick) and takes the linear interpolant
 * sum_i lambda_i s_i of the owner's element containing it; rendering,
 * classification, early termination, opacity correction and compositing are
 * those of vr_render_frame (sort-last mode only). Device memory: 80 bytes per
 * element (record + neighbours) plus 32 bytes per BVH node. */
vr_status vr_mesh_create(vr_ctx ctx, const int dims[3], const vr_partition *part, const float *verts,
                         long long n_verts, const float *values, const int *tets, long long n_tets,
                         vr_mesh *out);
vr_status vr_mesh_release(vr_mesh mesh);
/* Number of bricks, elements per brick (n long longs, may be NULL) and device
 * bytes of the mesh (may be NULL). */
vr_status vr_mesh_info(vr_mesh mesh, int *n_bricks, long long *elements_per_brick, long long *device_bytes);
/* One frame of the mesh with the context's camera, transfer function and
 * parameters: per-brick partials (BVH point location of each ray's first owned
 * sample, then a walk through face neighbours), then the composite, into
 * out_rgba (H x W x 4 float32; device if out_on_device, else host). Asynchronous
 * on `stream` like vr_render_frame. VR_ERR_STATE in ray-state cycling mode. */
vr_status vr_render_mesh_frame(vr_ctx ctx, vr_mesh mesh, float *out_rgba, int out_on_device, void *stream);

/* ---- fault injection (test hook) ----------------------------------------- */

/* For testing the error paths of the library and of its callers; the paper has
 * no counterpart. After `after` further successful device allocations (kind
 * VR_FAULT_ALLOC) or kernel launches (kind VR_FAULT_LAUNCH) made by the library
 * in this process, the next one fails on the host without calling CUDA: the
 * call in progress returns VR_ERR_OOM or VR_ERR_CUDA with a message naming the
 * injected fault, and the context and its objects stay usable. The plan is
 * one-shot and process-wide; VR_FAULT_NONE clears it. No GPU fault is raised:
 * nothing is launched or allocated in place of the failed operation.
 * VR_ERR_ARG for an unknown kind or a negative count. */
#define VR_FAULT_NONE 0
#define VR_FAULT_ALLOC 1
#define VR_FAULT_LAUNCH 2
vr_status vr_debug_inject_fault(int kind, int after);

/* ---- rendering without device allocation -------------------------------- */

/* The paper has no counterpart to this call; it exists for callers that must
 * not allocate device memory: a renderer embedded in a simulation that hands all
 * device memory to its own pool allocator (in-situ use), or a caller on a
 * latency-critical path where cudaMalloc/cudaFree, which synchronise the
 * device, are not allowed.
 *
 * Renders one frame (steps 1 + 2 of vr_render_frame, direct composite) from
 * caller-owned device memory: `volume_dev` is the x-fastest float32 volume of
 * dims[0] x dims[1] x dims[2] voxels, read in place (no packed bricks); the
 * image goes to `out_rgba_dev` (H x W x 4 float32, device). `tf_rgba` (n_tf
 * RGBA entries, 2 <= n_tf <= 1024) and `cam` are host memory. Nothing is
 * allocated on the device: the per-brick partial images, the composite's tile
 * masks and the transfer function live in one static device array of
 * VR_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits. A frame whose partial images (16 bytes per pixel of every
 * brick's footprint rectangle) and tile masks (16 bytes per 32 x 8 pixels)
 * would exceed it is rejected with VR_ERR_ARG before any device work.
 *   - Works on the current CUDA device. Every call looks up the scratch's
 *     device address (cudaGetSymbolAddress) on that device, so the call stays
 *     valid after a device reset; the first call on a device also loads the
 *     library's device code there, so make it before any stream capture.
 *   - All calls on a device share the scratch: calls that overlap on the GPU
 *     (other streams, other threads) race; order them on one stream. Each call
 *     rewrites every scratch byte it reads, so nothing needs clearing.
 *   - Asynchronous on `stream`; errors are returned as vr_status (no context,
 *     so no vr_last_error text). */
#define VR_NOALLOC_SCRATCH_BYTES (16u << 20)
vr_status vr_render_frame_noalloc(const float *volume_dev, const int dims[3], const vr_partition *part,
                                  const float *tf_rgba, int n_tf, float vmin, float vmax,
                                  const vr_camera *cam, float step_voxels, float ert_alpha,
                                  float *out_rgba_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* VR_H */
