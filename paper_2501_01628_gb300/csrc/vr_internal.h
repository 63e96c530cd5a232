// vr_internal.h -- structures shared by the host runtime (vr_host.cpp) and the
// CUDA kernels (vr_kernels.cu). Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/vr.h"

namespace vr {

constexpr int kMaxBricks = VR_MAX_BRICKS;

// Brick storage kind: the storage type and the cell layout -- xy-quads (four
// voxels of one plane per element; two loads per sample) or, for the 16-bit
// types, octets (both planes of a cell, 16 bytes per element; one load per
// sample). The first three equal vr_dtype's values.
enum StorageKind { kStoreF32 = 0, kStoreBF16 = 1, kStoreF16 = 2, kStoreBF16Oct = 3, kStoreF16Oct = 4 };
inline int storage_kind(vr_dtype t, bool octets) { return static_cast<int>(t) + (octets && t != VR_F32 ? 2 : 0); }
constexpr int kMaxFactors = 8;

// Work item of the no-allocation march: 16 x 8 pixels per 128-thread block,
// four 8 x 4 warp packets (the other marches take the packet width as a
// parameter, MarchParams::pw).
constexpr int kTileW = 16;
constexpr int kTileH = 8;
// Composite: 256-thread blocks of 32 x 8 threads, one thread per pixel of a
// 32 x 8 image tile with one brick mask per tile (the composite adjoint takes the
// same tiles).
constexpr int kCompW = 32;
constexpr int kCompH = 8;
constexpr int kCompTileH = kCompH;  // forward composite tile: kCompW x kCompTileH pixels
constexpr int kMaskThreads = 128;                // threads (tiles) per block of the tile-mask pass

// Brick storage index of quad (i, j, k): quads are grouped in 2x2x2 blocks of
// 128 bytes (one L1 line for float32), blocks x-fastest; nbx, nby = blocks per
// row and per plane. A warp's 8x4 ray packet then touches about the same
// number of lines whatever the view direction.
__host__ __device__ __forceinline__ int quad_index(int i, int j, int k, int nbx, int nby)
{
    return ((((k >> 1) * nby + (j >> 1)) * nbx + (i >> 1)) << 3) | ((k & 1) << 2) | ((j & 1) << 1) | (i & 1);
}

// Per-brick data of one frame, as the march kernel needs it.
struct BrickLaunch {
    int lo[3], hi[3];   // voxel box, half-open
    float own_lo[3];    // ownership bounds in voxel units (-inf / +inf on volume faces)
    float own_hi[3];
    int sx, sy;         // haloed brick extents in x and y (elements)
    long long base;     // quad offset of the brick's haloed xy-quad storage
    int rect[4];        // x0, y0, w, h of the footprint rectangle
    long long poff;     // float4 offset of the brick's partial
    int item_begin;     // first work item (tile) of this brick
    int tiles_x;        // tiles per rectangle row
};

// Everything one march launch needs; passed by value as the kernel parameter.
struct MarchParams {
    // camera, all FP32 (basis computed on the host in FP64)
    float eye[3], r[3], u[3], f[3];
    float tanx, tany;   // perspective: tan(fovy/2)*W/H, tan(fovy/2)
    float ow, oh;       // orthographic image-plane extent
    int ortho;
    int W, H;
    float inv_W, inv_H;  // 1/W, 1/H
    int pw;              // ray packet: a warp marches pw x (32/pw) pixels (pw = 4, 8 or 16)
    int tile_w, tile_h;  // work item: 2 x 2 packets = (2 pw) x (64/pw) pixels
    // volume
    float nmax;         // voxels per world unit
    float N[3];         // volume extent in voxels
    float dt, inv_dt;   // sample spacing (world units) and its inverse
    float ert_T;        // terminate a brick when T <= ert_T (negative: never)
    float opc_ratio;    // opacity correction step / reference step (1: off)
    // classification
    float tf_scale, tf_bias;  // x = s*scale + bias = (s - vmin)/(vmax - vmin)*(ntf-1)
    int ntf;
    const float4 *tf;   // 2*ntf float4: (T[i], T[i+1]-T[i]) pairs, last difference 0
    const void *data;   // brick storage
    float4 *partials;   // partial pool
    unsigned long long *sample_counter;  // non-null: count executed samples
    int *count_error;   // device error word; bit 4: in a counting launch, an executed
                        // sample's quad index fell outside its brick's storage
    // composite tile masks written by the first mask_blocks blocks of the
    // march grid (null: none): bit j of tile t's mask = the brick at visibility
    // position j overlaps composite tile t (kCompW x kCompTileH pixels)
    uint4 *tile_mask;
    int mask_tiles_x, mask_tiles_y, mask_blocks;
    // pipelined frames: the partial pool this frame writes was last read by the
    // composite of frame pool_frame - 2, which sets pool_done[pool] to its own
    // frame number when it is done; the march blocks wait for that (null: no
    // wait) before storing their partials
    const unsigned long long *pool_done;
    unsigned long long pool_frame;
    int pool;
    int nb;
    int n_items;        // march work items (the grid adds mask_blocks in front)
    int order[kMaxBricks];  // brick ids front to back (ray-state cycling)
    BrickLaunch b[kMaxBricks];
};

struct CompositeParams {
    int W, H;
    int nb;
    int n_levels;                     // 1 = direct
    int order[kMaxBricks];            // brick ids front to back
    unsigned long long gid[kMaxBricks + 1];   // radix-k: byte l-1 = group index of position q at level l
                                              // (entry nb: one past the last group at every level)
    int rect[kMaxBricks][4];          // by brick id
    long long poff[kMaxBricks];       // by brick id
    const float4 *partials;
    float4 *out;
    uint4 *tile_mask;                 // per tile: visibility positions of the bricks overlapping it
    int tiles_x, tiles_y;             // composite tiles per row / column (kCompW x kCompTileH)
    // pipelined frames: the grid's last block to finish sets pool_done[pool] =
    // pool_frame (pool_count counts finished blocks; null: nothing published)
    unsigned long long *pool_done;
    unsigned int *pool_count;
    unsigned long long pool_frame;
    int pool;
};

// Composite adjoint: the composite's layout plus the image gradient and the
// per-brick partial gradients it produces (same layout as the partials).
struct CompositeGradParams {
    int W, H;
    int nb;
    int order[kMaxBricks];
    int rect[kMaxBricks][4];
    long long poff[kMaxBricks];
    const float4 *partials;
    const float4 *grad_img;
    float4 *grad_partials;
};

// March adjoint outputs (gradients are added into).
struct GradArgs {
    const float4 *grad_partials;
    float *grad_tf;   // ntf x 4
    float *grad_vol;  // Nz x Ny x Nx, or null
    int N[3];
    int *error;       // device error word: bit 0 = a run exceeded the checkpoint storage
};

// Batched form: per view, the camera fields that dev::owned_run reads (same
// names as MarchParams) and the view's work-item counts.
struct BatchView {
    float eye[3], r[3], u[3], f[3];
    float tanx, tany;
    float ow, oh;
    int ortho;
    int W, H;
    float inv_W, inv_H;
    float nmax;
    float N[3];
    float dt, inv_dt;
    int march_items;  // (brick, tile) items of one render of this view
    int comp_items;   // composite tiles of one render of this view
};

constexpr int kBatchCompW = 16;  // composite tile of the batched kernel (128 threads)
constexpr int kBatchCompH = 8;

struct BatchParams {
    int n_renders, n_views, nb;
    int mode;                        // 0: unit = one render; 1: unit = one volume, all views, brick-major
    int n_units;
    const int *unit_march;           // per unit: march items
    const int *unit_comp;            // per unit: composite tiles
    const long long *bw_begin;       // mode 1: nb x n_views + 1 tile offsets, (brick, view) order
    long long view_stride;           // mode 1: partial pixels per view inside a unit's ring slot
    int pw;                          // ray-packet width: a warp marches pw x (32/pw) pixels
    long long total_items;
    const long long *render_begin;   // n_units + 2 segment starts: segment g = march items of
                                     // unit g, then composite tiles of unit g-1
    const BatchView *views;          // n_views
    const BrickLaunch *vb;           // n_views x nb; rect/poff/item_begin/tiles_x per view
    const int *order;                // n_views x nb, front to back
    const void *const *vol_data;     // per volume: brick storage
    const float2 *vol_tf;            // per volume: (tf_scale, tf_bias)
    const float4 *tf;                // (T, dT) pairs
    int ntf;
    float ert_T;
    float opc_ratio;                 // opacity correction (1: off)
    float4 *ring;                    // slots x slot_px partial pixels
    long long slot_px;               // partial pixels per ring slot (one unit)
    int slots;
    float4 *out;                     // n_renders x H x W
    unsigned long long *claim;       // work counter
    int *march_done;                 // per unit: finished march items
    int *comp_done;                  // per unit: finished composite tiles
    int *error;                      // bit 1: a bounded wait gave up
    int wait_limit;                  // spin iterations (about 128 ns each) before giving up
    int wait_extra;                  // added to unit 0's march target by composite waits (test hook; 0)
};

// "over" of n images, front to back, pixel by pixel (vr_composite_images).
struct ImagesParams {
    const float4 *img[kMaxBricks];
    int n;
    long long pixels;
    float4 *out;
};

// Pack of all bricks of a volume in one launch: block j of brick b (counted
// from that brick's block_begin) writes the brick's storage quads
// [j*kPackChunk, (j+1)*kPackChunk), in storage order.
constexpr int kPackChunk = 2048;
struct PackBrick {
    void *dst;             // the brick's storage
    long long quads;       // quads in the brick's storage (whole 2x2x2 blocks)
    int lo[3];             // voxel box origin
    int s[3];              // haloed extents (the brick stores (s0-1)(s1-1)s2 quads)
    int block_begin;       // first block of this brick
    int row;               // scalar copies: padded row length in elements (multiple of 4)
};
struct PackParams {
    const float *src;      // x-fastest float32 volume
    int N[3];
    int nb;
    int n_blocks;
    PackBrick b[kMaxBricks];
};

// Staged march (vr_staged.cu): scalar copies of the bricks, haloed, rows padded
// to a multiple of 4 elements; kStageCap floats per shared-memory stage (two
// stages per block).
constexpr int kStageCap = 4096;
struct StagedBricks {
    const float *scalar;          // all bricks' scalar copies
    long long sbase[kMaxBricks];  // element offset of each brick (a multiple of 32)
    int sxp[kMaxBricks];          // padded row length (elements)
};

// Launchers (vr_kernels.cu). They return the launch's cudaError_t.
// `kind` is a StorageKind.
cudaError_t launch_pack(const PackParams &p, int kind, cudaStream_t s);
// after_composite: launch as a programmatic dependent of the preceding kernel
// (the previous pipelined frame's composite); see march_kernel.
cudaError_t launch_march(const MarchParams &p, int kind, cudaStream_t s, bool after_composite = false);
// after_frame: launch as a programmatic dependent of the preceding kernel (the
// previous pipelined frame); see march_cycle_kernel.
cudaError_t launch_march_cycle(const MarchParams &p, int kind, float4 *out, cudaStream_t s, bool after_frame = false);
// max_blocks > 0: a grid of at most that many blocks, each compositing tiles in
// turn; 0: one block per tile.
cudaError_t launch_composite(const CompositeParams &p, cudaStream_t s, int max_blocks = 0);
cudaError_t launch_composite_images(const ImagesParams &p, cudaStream_t s);
// Tile masks of p (p.tile_mask) for frames whose march did not write them.
cudaError_t launch_tile_masks(const CompositeParams &p, cudaStream_t s);
cudaError_t launch_composite_grad(const CompositeGradParams &p, cudaStream_t s);
cudaError_t launch_march_grad(const MarchParams &p, const GradArgs &g, int kind, cudaStream_t s);
// Persistent batched kernel: cooperative launch of `blocks` blocks of 128 threads.
cudaError_t launch_batch(const BatchParams &p, int kind, int blocks, cudaStream_t s);
int batch_max_blocks_per_sm(int kind);
// Staged march and the scalar brick pack (vr_staged.cu).
cudaError_t launch_march_staged(const MarchParams &p, const StagedBricks &sb, cudaStream_t s);
cudaError_t launch_scalar_pack(const PackParams &p, cudaStream_t s);

}  // namespace vr
