// vr_host.cpp -- host runtime of libvr: contexts, brick partitions and their
// kd visibility trees, per-view footprint rectangles and launch tables, and the
// C ABI declared in include/vr.h.
//
// Sec. 2.2 of arXiv:2501.01628: data is spatially distributed over ranks
// (here: bricks on one GPU); the distribution may be uneven (Sec. 4).
// Sec. 3: rendering is one collective call whose image ends up in one
// framebuffer; the world is distributed and updated locally.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "vr_objects.h"

using namespace vr;
using namespace vr::host;

namespace vr {
namespace host {

// ---- fault injection (vr_debug_inject_fault) --------------------------------
std::atomic<int> g_fault_kind{VR_FAULT_NONE};
std::atomic<long long> g_fault_after{0};

bool fault_now(int kind)
{
    if (g_fault_kind.load(std::memory_order_relaxed) != kind) return false;
    if (g_fault_after.fetch_sub(1) > 0) return false;
    g_fault_kind.store(VR_FAULT_NONE);
    return true;
}

size_t elem_size(vr_dtype t) { return t == VR_F32 ? 4 : 2; }
// bytes of one xy-quad (four voxels) in device storage
// bytes of one storage element: an xy-quad (four voxels), or an octet (both
// planes of a cell, 16-bit types only)
size_t quad_size(vr_dtype t, bool octets) { return (octets && t != VR_F32 ? 8 : 4) * elem_size(t); }
// quads stored for a brick: haloed extents (sx, sy, sz) give (sx-1) x (sy-1) x sz
// quads, rounded up to whole 2x2x2 blocks
long long brick_quads(const int *bx)
{
    const long long nbx = (bx[3] - bx[0] + 2) / 2, nby = (bx[4] - bx[1] + 2) / 2,
                    nbz = (bx[5] - bx[2] + 3) / 2;
    return nbx * nby * nbz * 8;
}

vr_status fail(vr_ctx ctx, vr_status s, const std::string &msg)
{
    if (ctx) ctx->last_error = msg;
    return s;
}

vr_status cuda_fail(vr_ctx ctx, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? VR_ERR_OOM : VR_ERR_CUDA, m);
}

int nmax3(const int d[3]) { return std::max(d[0], std::max(d[1], d[2])); }

// ---- partitions -----------------------------------------------------------

bool grid_boxes(const int dims[3], const int g[3], std::vector<int> &boxes)
{
    for (int a = 0; a < 3; ++a)
        if (g[a] < 1 || g[a] > dims[a]) return false;
    boxes.clear();
    for (int bz = 0; bz < g[2]; ++bz)
        for (int by = 0; by < g[1]; ++by)
            for (int bx = 0; bx < g[0]; ++bx) {
                const int b[3] = {bx, by, bz};
                int lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    lo[a] = static_cast<int>((static_cast<long long>(dims[a]) * b[a]) / g[a]);
                    hi[a] = static_cast<int>((static_cast<long long>(dims[a]) * (b[a] + 1)) / g[a]);
                }
                boxes.insert(boxes.end(), {lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]});
            }
    return true;
}

bool kd_boxes(const int dims[3], int n, const double *u, std::vector<int> &boxes)
{
    if (n < 1 || (n > 1 && !u)) return false;
    boxes.assign(6 * static_cast<size_t>(n), 0);
    boxes[3] = dims[0];
    boxes[4] = dims[1];
    boxes[5] = dims[2];
    for (int count = 1; count < n; ++count) {
        int best = 0;
        long long bestv = -1;
        for (int l = 0; l < count; ++l) {
            const int *b = &boxes[6 * l];
            long long v = static_cast<long long>(b[3] - b[0]) * (b[4] - b[1]) * (b[5] - b[2]);
            if (v > bestv) {
                bestv = v;
                best = l;
            }
        }
        int *b = &boxes[6 * best];
        int axis = 0;
        for (int a = 1; a < 3; ++a)
            if (b[3 + a] - b[a] > b[3 + axis] - b[axis]) axis = a;
        const int ext = b[3 + axis] - b[axis];
        if (ext < 2 || !(u[count - 1] >= 0.0 && u[count - 1] <= 1.0)) return false;
        int cut = b[axis] + static_cast<int>(std::floor(u[count - 1] * ext + 0.5));
        cut = std::min(std::max(cut, b[axis] + 1), b[3 + axis] - 1);
        int *nbx = &boxes[6 * count];
        std::memcpy(nbx, b, 6 * sizeof(int));
        b[3 + axis] = cut;
        nbx[axis] = cut;
    }
    return true;
}

// Builds a kd tree over `ids` (boxes inside `region`) by finding axis-aligned
// planes that separate the boxes; fails if the boxes do not tile the region or
// admit no such plane. Front-to-back order is then a tree traversal.
bool build_tree(const std::vector<int> &boxes, std::vector<int> ids, const int region[6],
                std::vector<KdNode> &tree, int &node_out)
{
    node_out = static_cast<int>(tree.size());
    tree.emplace_back();
    if (ids.size() == 1) {
        const int *b = &boxes[6 * ids[0]];
        for (int i = 0; i < 6; ++i)
            if (b[i] != region[i]) return false;
        tree[node_out].brick = ids[0];
        return true;
    }
    for (int axis = 0; axis < 3; ++axis) {
        std::vector<int> cands;
        for (int id : ids) cands.push_back(boxes[6 * id + axis]);
        std::sort(cands.begin(), cands.end());
        cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
        for (int c : cands) {
            if (c <= region[axis] || c >= region[3 + axis]) continue;
            std::vector<int> lo_ids, hi_ids;
            bool ok = true;
            for (int id : ids) {
                const int *b = &boxes[6 * id];
                if (b[3 + axis] <= c) lo_ids.push_back(id);
                else if (b[axis] >= c) hi_ids.push_back(id);
                else {
                    ok = false;
                    break;
                }
            }
            if (!ok || lo_ids.empty() || hi_ids.empty()) continue;
            int rlo[6], rhi[6];
            std::memcpy(rlo, region, sizeof(rlo));
            std::memcpy(rhi, region, sizeof(rhi));
            rlo[3 + axis] = c;
            rhi[axis] = c;
            int a = -1, b = -1;
            if (!build_tree(boxes, lo_ids, rlo, tree, a)) return false;
            if (!build_tree(boxes, hi_ids, rhi, tree, b)) return false;
            tree[node_out].axis = axis;
            tree[node_out].cut = c;
            tree[node_out].child[0] = a;
            tree[node_out].child[1] = b;
            return true;
        }
    }
    return false;
}

void visibility_order(const std::vector<KdNode> &tree, int node, const vr_camera &cam, double nmax,
                      std::vector<int> &out)
{
    const KdNode &n = tree[node];
    if (n.axis < 0) {
        out.push_back(n.brick);
        return;
    }
    bool low_first;
    if (cam.ortho) low_first = cam.dir[n.axis] >= 0.0;
    else low_first = cam.eye[n.axis] * nmax <= static_cast<double>(n.cut);
    visibility_order(tree, n.child[low_first ? 0 : 1], cam, nmax, out);
    visibility_order(tree, n.child[low_first ? 1 : 0], cam, nmax, out);
}

void normalize(double v[3])
{
    const double l = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= l;
    v[1] /= l;
    v[2] /= l;
}

void cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

bool make_basis(const vr_camera &c, Basis &B)
{
    for (int i = 0; i < 3; ++i) B.f[i] = c.dir[i];
    if (B.f[0] == 0 && B.f[1] == 0 && B.f[2] == 0) return false;
    normalize(B.f);
    cross(c.up, B.f, B.r);
    if (B.r[0] == 0 && B.r[1] == 0 && B.r[2] == 0) return false;
    normalize(B.r);
    cross(B.f, B.r, B.u);
    const double th = std::tan(c.fovy_deg * M_PI / 360.0);
    B.tany = th;
    B.tanx = th * static_cast<double>(c.width) / c.height;
    return true;
}

// Conservative pixel rectangle of a brick's projected bounding box (+1 px).
void footprint(const vr_camera &c, const Basis &B, const int box[6], double nmax, int rect[4])
{
    const int W = c.width, H = c.height;
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    int behind = 0;
    for (int k = 0; k < 8; ++k) {
        double q[3], v[3];
        for (int a = 0; a < 3; ++a) {
            q[a] = ((k >> a) & 1 ? box[3 + a] : box[a]) / nmax;
            v[a] = q[a] - c.eye[a];
        }
        const double vr = v[0] * B.r[0] + v[1] * B.r[1] + v[2] * B.r[2];
        const double vu = v[0] * B.u[0] + v[1] * B.u[1] + v[2] * B.u[2];
        double x, y;
        if (c.ortho) {
            x = (vr / c.ortho_w + 0.5) * W - 0.5;
            y = (vu / c.ortho_h + 0.5) * H - 0.5;
        } else {
            const double z = v[0] * B.f[0] + v[1] * B.f[1] + v[2] * B.f[2];
            if (z <= 1e-9) {
                ++behind;
                continue;
            }
            x = (vr / (z * B.tanx) + 1.0) * 0.5 * W - 0.5;
            y = (vu / (z * B.tany) + 1.0) * 0.5 * H - 0.5;
        }
        xmin = std::min(xmin, x);
        xmax = std::max(xmax, x);
        ymin = std::min(ymin, y);
        ymax = std::max(ymax, y);
    }
    if (behind == 8) {
        rect[0] = rect[1] = rect[2] = rect[3] = 0;
        return;
    }
    if (behind > 0) {
        rect[0] = 0;
        rect[1] = 0;
        rect[2] = W;
        rect[3] = H;
        return;
    }
    const double x0 = std::max(0.0, std::floor(xmin) - 1.0), x1 = std::min(W - 1.0, std::ceil(xmax) + 1.0);
    const double y0 = std::max(0.0, std::floor(ymin) - 1.0), y1 = std::min(H - 1.0, std::ceil(ymax) + 1.0);
    if (x1 < x0 || y1 < y0) {
        rect[0] = rect[1] = rect[2] = rect[3] = 0;
        return;
    }
    rect[0] = static_cast<int>(x0);
    rect[1] = static_cast<int>(y0);
    rect[2] = static_cast<int>(x1 - x0) + 1;
    rect[3] = static_cast<int>(y1 - y0) + 1;
}

// Boxes + kd tree of a partition description; false (with a reason) if invalid.
bool partition_plan(const int dims[3], const vr_partition *part, std::vector<int> &boxes,
                    std::vector<KdNode> &tree, const char **why)
{
    *why = "invalid partition description";
    if (!dims || !part) return false;
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || dims[a] > (1 << 16)) {
            *why = "bad volume dims";
            return false;
        }
    bool ok = false;
    switch (part->kind) {
    case VR_PART_GRID: ok = grid_boxes(dims, part->grid, boxes); break;
    case VR_PART_KD: ok = kd_boxes(dims, part->n_bricks, part->cut_fracs, boxes); break;
    case VR_PART_BOXES:
        if (part->boxes && part->n_bricks >= 1 && part->n_bricks <= kMaxBricks) {
            boxes.assign(part->boxes, part->boxes + 6 * static_cast<size_t>(part->n_bricks));
            ok = true;
        }
        break;
    default: break;
    }
    if (!ok) return false;
    const int nb = static_cast<int>(boxes.size() / 6);
    if (nb > kMaxBricks) {
        *why = "too many bricks";
        return false;
    }
    for (int b = 0; b < nb; ++b)
        for (int a = 0; a < 3; ++a) {
            const int lo = boxes[6 * b + a], hi = boxes[6 * b + 3 + a];
            if (lo < 0 || hi > dims[a] || lo >= hi) {
                *why = "brick box out of range";
                return false;
            }
        }
    std::vector<int> ids(nb);
    for (int b = 0; b < nb; ++b) ids[b] = b;
    const int region[6] = {0, 0, 0, dims[0], dims[1], dims[2]};
    int root = -1;
    tree.clear();
    if (!build_tree(boxes, ids, region, tree, root)) {
        *why = "bricks do not tile the volume with axis-aligned cuts";
        return false;
    }
    return true;
}

bool camera_valid(const vr_camera *cam)
{
    if (!cam || cam->width < 1 || cam->height < 1 || cam->width > 32768 || cam->height > 32768) return false;
    if (cam->ortho ? !(cam->ortho_w > 0 && cam->ortho_h > 0) : !(cam->fovy_deg > 0 && cam->fovy_deg < 180))
        return false;
    Basis B;
    return make_basis(*cam, B);
}

// Pack every brick of `vol` from the device float32 volume `dsrc`.
cudaError_t pack_bricks(vr_volume vol, const float *dsrc, cudaStream_t s)
{
    vol->ctx->input_seq++;  // a pipelined march must not overlap this pack
    const size_t es = quad_size(vol->dtype, vol->octets);
    const int nb = static_cast<int>(vol->boxes.size() / 6);
    static thread_local PackParams pp;
    pp.src = dsrc;
    for (int a = 0; a < 3; ++a) pp.N[a] = vol->dims[a];
    pp.nb = nb;
    long long blocks = 0;
    for (int b = 0; b < nb; ++b) {
        const int *bx = &vol->boxes[6 * b];
        PackBrick &B = pp.b[b];
        B.dst = static_cast<char *>(vol->d_data) + vol->base[b] * static_cast<long long>(es);
        B.quads = vol->holds(b) ? brick_quads(bx) : 0;
        for (int a = 0; a < 3; ++a) {
            B.lo[a] = bx[a];
            B.s[a] = bx[3 + a] - bx[a] + 2;
        }
        B.block_begin = static_cast<int>(blocks);
        B.row = 0;
        blocks += (B.quads + kPackChunk - 1) / kPackChunk;
    }
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    pp.n_blocks = static_cast<int>(blocks);
    if (fault_now(VR_FAULT_LAUNCH)) return cudaErrorLaunchFailure;
    cudaError_t e = launch_pack(pp, vol->kind(), s);
    if (e != cudaSuccess || !vol->d_scalar) return e;
    // the staged march's scalar copy
    blocks = 0;
    for (int b = 0; b < nb; ++b) {
        PackBrick &B = pp.b[b];
        B.dst = vol->d_scalar + vol->sbase[b];
        B.row = vol->sxp[b];
        B.quads = vol->holds(b) ? static_cast<long long>(B.row) * B.s[1] * B.s[2] : 0;
        B.block_begin = static_cast<int>(blocks);
        blocks += (B.quads + kPackChunk - 1) / kPackChunk;
    }
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    pp.n_blocks = static_cast<int>(blocks);
    if (fault_now(VR_FAULT_LAUNCH)) return cudaErrorLaunchFailure;
    return launch_scalar_pack(pp, s);
}

vr_status ensure_frame(vr_ctx ctx, vr_frame_s &fr, long long px)
{
    if (px <= fr.cap_px) return VR_OK;
    const long long want = std::max(px, fr.cap_px + fr.cap_px / 4);
    if (fr.d_part) cudaFree(fr.d_part);
    fr.d_part = nullptr;
    fr.cap_px = 0;
    VR_CUDA(ctx, vr::host::dev_malloc(&fr.d_part, static_cast<size_t>(want) * sizeof(float4)));
    fr.cap_px = want;
    return VR_OK;
}

// Per-view setup (host, tiny): visibility order, footprints, launch table.
vr_status prepare_frame(vr_ctx ctx, vr_volume vol, vr_frame_s &fr, MarchParams &mp)
{
    if (!ctx->has_cam) return fail(ctx, VR_ERR_STATE, "no camera set");
    if (!ctx->has_tf) return fail(ctx, VR_ERR_STATE, "no transfer function set");
    const vr_camera &c = ctx->cam;
    Basis B;
    if (!make_basis(c, B)) return fail(ctx, VR_ERR_ARG, "degenerate camera basis");
    const int nb = static_cast<int>(vol->boxes.size() / 6);
    const double nmax = nmax3(vol->dims);
    fr.ctx = ctx;
    fr.nb = nb;
    fr.W = c.width;
    fr.H = c.height;
    fr.rects.assign(4 * nb, 0);
    fr.poff.assign(nb, 0);
    fr.order.clear();
    visibility_order(vol->tree, 0, c, nmax, fr.order);
    long long px = 0;
    int items = 0;
    std::memset(&mp, 0, sizeof(mp));
    const int pw = ctx->packet_width, tile_w = 2 * pw, tile_h = 2 * (32 / pw);
    mp.pw = pw;
    mp.tile_w = tile_w;
    mp.tile_h = tile_h;
    for (int b = 0; b < nb; ++b) {
        int *r = &fr.rects[4 * b];
        footprint(c, B, &vol->boxes[6 * b], nmax, r);
        if (!vol->holds(b)) r[0] = r[1] = r[2] = r[3] = 0;  // not in this share: an empty partial
        fr.poff[b] = px;
        px += static_cast<long long>(r[2]) * r[3];
        px = (px + 7) & ~7LL;  // 128-byte aligned partial starts
        BrickLaunch &L = mp.b[b];
        const int *bx = &vol->boxes[6 * b];
        for (int a = 0; a < 3; ++a) {
            L.lo[a] = bx[a];
            L.hi[a] = bx[3 + a];
            L.own_lo[a] = bx[a] == 0 ? -INFINITY : static_cast<float>(bx[a]);
            L.own_hi[a] = bx[3 + a] == vol->dims[a] ? INFINITY : static_cast<float>(bx[3 + a]);
        }
        L.sx = bx[3] - bx[0] + 2;
        L.sy = bx[4] - bx[1] + 2;
        L.base = vol->base[b];
        std::memcpy(L.rect, r, sizeof(L.rect));
        L.poff = fr.poff[b];
        L.item_begin = items;
        L.tiles_x = (r[2] + tile_w - 1) / tile_w;
        const int tiles_y = (r[3] + tile_h - 1) / tile_h;
        items += L.tiles_x * tiles_y;
    }
    fr.total_px = px;
    fr.tiles_x = (c.width + kCompW - 1) / kCompW;
    fr.tiles_y = (c.height + kCompTileH - 1) / kCompTileH;
    fr.pool_px = px + static_cast<long long>(fr.tiles_x) * fr.tiles_y;
    fr.masks_ready = false;
    for (int a = 0; a < 3; ++a) {
        mp.eye[a] = static_cast<float>(c.eye[a]);
        mp.r[a] = static_cast<float>(B.r[a]);
        mp.u[a] = static_cast<float>(B.u[a]);
        mp.f[a] = static_cast<float>(B.f[a]);
        mp.N[a] = static_cast<float>(vol->dims[a]);
    }
    mp.tanx = static_cast<float>(B.tanx);
    mp.tany = static_cast<float>(B.tany);
    mp.ow = static_cast<float>(c.ortho_w);
    mp.oh = static_cast<float>(c.ortho_h);
    mp.ortho = c.ortho ? 1 : 0;
    mp.W = c.width;
    mp.H = c.height;
    mp.inv_W = static_cast<float>(1.0 / c.width);
    mp.inv_H = static_cast<float>(1.0 / c.height);
    mp.nmax = static_cast<float>(nmax);
    const double dt = static_cast<double>(ctx->step) / nmax;
    mp.dt = static_cast<float>(dt);
    mp.inv_dt = static_cast<float>(1.0 / dt);
    mp.ert_T = ctx->ert_alpha < 1.0f ? static_cast<float>(1.0 - static_cast<double>(ctx->ert_alpha)) : -1.0f;
    mp.opc_ratio = ctx->opc_ref > 0.0f ? static_cast<float>(static_cast<double>(ctx->step) / ctx->opc_ref) : 1.0f;
    {
        const double scale = (ctx->ntf - 1) / (static_cast<double>(ctx->vmax) - ctx->vmin);
        mp.tf_scale = static_cast<float>(scale);
        mp.tf_bias = static_cast<float>(-static_cast<double>(ctx->vmin) * scale);
    }
    mp.ntf = ctx->ntf;
    mp.tf = ctx->d_tf;
    mp.data = vol->d_data;
    mp.sample_counter = ctx->count_samples ? ctx->d_counter : nullptr;
    mp.count_error = ctx->d_error;
    mp.nb = nb;
    mp.n_items = items;
    for (int j = 0; j < nb; ++j) mp.order[j] = fr.order[j];
    return VR_OK;
}

cudaEvent_t pooled_event(vr_ctx ctx)
{
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Records the start event of a timed launch; returns the index or -1.
int timing_begin(vr_ctx ctx, int kind, cudaStream_t s)
{
    if (!ctx->timing) return -1;
    cudaEvent_t a = pooled_event(ctx), b = pooled_event(ctx);
    if (!a || !b || cudaEventRecord(a, s) != cudaSuccess) {
        if (a) ctx->event_pool.push_back(a);
        if (b) ctx->event_pool.push_back(b);
        return -1;
    }
    ctx->timed.push_back({a, b, kind});
    return static_cast<int>(ctx->timed.size()) - 1;
}

void timing_end(vr_ctx ctx, int idx, cudaStream_t s)
{
    if (idx >= 0) cudaEventRecord(ctx->timed[idx].b, s);
}

vr_status march(vr_ctx ctx, vr_volume vol, vr_frame_s &fr, cudaStream_t s, bool after_composite = false,
                const PoolSync *sync = nullptr)
{
    static thread_local MarchParams mp;  // ~12 KB: keep off the stack
    vr_status st = prepare_frame(ctx, vol, fr, mp);
    if (st != VR_OK) return st;
    st = ensure_frame(ctx, fr, std::max(fr.pool_px, 1LL));
    if (st != VR_OK) return st;
    mp.partials = fr.d_part;
    // the march grid's first blocks write the composite's tile masks
    mp.tile_mask = reinterpret_cast<uint4 *>(fr.d_part + fr.total_px);
    mp.mask_tiles_x = fr.tiles_x;
    mp.mask_tiles_y = fr.tiles_y;
    mp.mask_blocks = (fr.tiles_x * fr.tiles_y + kMaskThreads - 1) / kMaskThreads;
    if (sync) {
        mp.pool_done = sync->done;
        mp.pool_frame = sync->frame;
        mp.pool = sync->pool;
    }
    const int t = timing_begin(ctx, 0, s);
    if (ctx->staging && vol->d_scalar) {
        static thread_local StagedBricks sb;
        sb.scalar = vol->d_scalar;
        for (size_t b = 0; b < vol->sbase.size(); ++b) {
            sb.sbase[b] = vol->sbase[b];
            sb.sxp[b] = vol->sxp[b];
        }
        VR_LAUNCH(ctx, launch_march_staged(mp, sb, s));
    } else {
        VR_LAUNCH(ctx, launch_march(mp, vol->kind(), s, after_composite));
    }
    timing_end(ctx, t, s);
    fr.masks_ready = true;
    return VR_OK;
}

vr_status composite(vr_ctx ctx, vr_frame_s &fr, float4 *out, cudaStream_t s, int max_blocks = 0,
                    const PoolSync *sync = nullptr)
{
    static thread_local CompositeParams cp;
    std::memset(&cp, 0, sizeof(cp));
    cp.W = fr.W;
    cp.H = fr.H;
    cp.nb = fr.nb;
    const int nf = static_cast<int>(ctx->factors.size());
    long long prod = 1;
    for (int k : ctx->factors) prod *= k;
    const bool radix = nf > 0 && prod == fr.nb;
    if (nf > 0 && !radix)
        return fail(ctx, VR_ERR_ARG, "composite schedule factors do not multiply to the brick count");
    cp.n_levels = radix ? nf : 1;
    // gid[q]: the group of visibility position q at each level l >= 1 of the
    // association tree (groups of factors[0] x ... x factors[l-1] positions)
    for (int j = 0; j < fr.nb; ++j) cp.order[j] = fr.order[j];
    for (int q = 0; q <= fr.nb; ++q) {
        unsigned long long g = 0;
        long long size = 1;
        for (int l = 1; l < cp.n_levels; ++l) {
            size *= ctx->factors[l - 1];
            g |= static_cast<unsigned long long>((q / size) & 0xff) << (8 * (l - 1));
        }
        cp.gid[q] = g;
    }
    for (int b = 0; b < fr.nb; ++b) {
        std::memcpy(cp.rect[b], &fr.rects[4 * b], 4 * sizeof(int));
        cp.poff[b] = fr.poff[b];
    }
    cp.partials = fr.d_part;
    cp.out = out;
    cp.tile_mask = reinterpret_cast<uint4 *>(fr.d_part + fr.total_px);
    cp.tiles_x = fr.tiles_x;
    cp.tiles_y = fr.tiles_y;
    if (!fr.masks_ready) {  // a march that does not write them (meshes)
        VR_LAUNCH(ctx, launch_tile_masks(cp, s));
        fr.masks_ready = true;
    }
    const int t = timing_begin(ctx, 1, s);
    if (sync) {
        cp.pool_done = sync->done;
        cp.pool_count = sync->count;
        cp.pool_frame = sync->frame;
        cp.pool = sync->pool;
    }
    VR_LAUNCH(ctx, launch_composite(cp, s, max_blocks));
    timing_end(ctx, t, s);
    return VR_OK;
}

// Staging image for a host output. Synchronous mode: one buffer, the caller's
// stream waits for the copy. Asynchronous mode: two buffers used in turn; the
// render stream first waits until the buffer's previous copy is done.
vr_status host_staging(vr_ctx ctx, long long px, cudaStream_t s, float4 **buf, int *slot)
{
    if (!ctx->host_async) {
        if (px > ctx->img_cap) {
            if (ctx->d_img) cudaFree(ctx->d_img);
            ctx->d_img = nullptr;
            ctx->img_cap = 0;
            VR_CUDA(ctx, vr::host::dev_malloc(&ctx->d_img, static_cast<size_t>(px) * sizeof(float4)));
            ctx->img_cap = px;
        }
        *buf = ctx->d_img;
        *slot = -1;
        return VR_OK;
    }
    if (!ctx->copy_stream) {
        VR_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            VR_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_rendered[i], cudaEventDisableTiming));
            VR_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_copied[i], cudaEventDisableTiming));
        }
    }
    if (px > ctx->img2_cap) {
        VR_CUDA(ctx, cudaStreamSynchronize(ctx->copy_stream));
        for (int i = 0; i < 2; ++i) {
            cudaFree(ctx->d_img2[i]);
            ctx->d_img2[i] = nullptr;
        }
        ctx->img2_cap = 0;
        for (int i = 0; i < 2; ++i)
            VR_CUDA(ctx, vr::host::dev_malloc(&ctx->d_img2[i], static_cast<size_t>(px) * sizeof(float4)));
        ctx->img2_cap = px;
    }
    const int k = ctx->img_next;
    ctx->img_next ^= 1;
    // The staging image is free once its previous copy (two frames back) is
    // done. Outside stream capture the host waits for that here, which keeps
    // the render stream free of wait nodes: a wait between a pipelined frame's
    // march and its composite would keep the composite from becoming resident
    // in the march's tail (and the next march from starting there).
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    VR_CUDA(ctx, cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusNone)
        VR_CUDA(ctx, cudaEventSynchronize(ctx->ev_copied[k]));
    else
        VR_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_copied[k], 0));
    *buf = ctx->d_img2[k];
    *slot = k;
    return VR_OK;
}

// Copy a staged image to host memory: at once and waiting (synchronous mode),
// or on the copy stream after the render (asynchronous mode; vr_sync waits).
vr_status host_copy(vr_ctx ctx, float *out, const float4 *buf, int slot, long long px, cudaStream_t s)
{
    const size_t bytes = static_cast<size_t>(px) * sizeof(float4);
    if (slot < 0) {
        VR_CUDA(ctx, cudaMemcpyAsync(out, buf, bytes, cudaMemcpyDeviceToHost, s));
        VR_CUDA(ctx, cudaStreamSynchronize(s));
        return VR_OK;
    }
    VR_CUDA(ctx, cudaEventRecord(ctx->ev_rendered[slot], s));
    VR_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_rendered[slot], 0));
    VR_CUDA(ctx, cudaMemcpyAsync(out, buf, bytes, cudaMemcpyDeviceToHost, ctx->copy_stream));
    VR_CUDA(ctx, cudaEventRecord(ctx->ev_copied[slot], ctx->copy_stream));
    return VR_OK;
}

vr_status composite_to(vr_ctx ctx, vr_frame_s &fr, float *out, int out_on_device, cudaStream_t s)
{
    if (!out) return fail(ctx, VR_ERR_ARG, "null output");
    const long long px = static_cast<long long>(fr.W) * fr.H;
    if (out_on_device) return composite(ctx, fr, reinterpret_cast<float4 *>(out), s);
    float4 *buf = nullptr;
    int slot = -1;
    vr_status st = host_staging(ctx, px, s, &buf, &slot);
    if (st != VR_OK) return st;
    st = composite(ctx, fr, buf, s);
    if (st != VR_OK) return st;
    return host_copy(ctx, out, buf, slot, px, s);
}

// Pipelined frames: whether this frame's first kernel may be launched as a
// programmatic dependent of the preceding kernel -- the previous pipelined
// frame was launched on the same stream and no brick pack or table upload of
// this context came since (input_seq). Until this frame's last kernel is
// launched (pipe_launched) no further frame may overlap.
bool pipe_after(vr_ctx ctx, cudaStream_t s)
{
    const bool after = ctx->pipe_ready && ctx->pipe_stream == s && ctx->pipe_seq == ctx->input_seq;
    ctx->pipe_ready = false;
    return after;
}

void pipe_launched(vr_ctx ctx, cudaStream_t s)
{
    ctx->pipe_ready = true;
    ctx->pipe_stream = s;
    ctx->pipe_seq = ctx->input_seq;
}

bool pipelined_output(vr_ctx ctx, int out_on_device)
{
    return ctx->pipelining && (out_on_device || ctx->host_async) && !ctx->timing;
}

// The next pipelined frame's number and pool (frame n uses pool n % 2; its
// march waits for the composite of frame n - 2, which read the same pool).
PoolSync pipe_frame(vr_ctx ctx)
{
    const unsigned long long n = ++ctx->pool_frame;
    return PoolSync{ctx->d_pool_done, ctx->d_pool_count, n, static_cast<int>(n & 1)};
}

vr_frame_s &pipe_pool(vr_ctx ctx, const PoolSync &sync)
{
    return sync.pool ? ctx->frame2 : ctx->frame;
}

// The composite of a pipelined frame: a persistent grid of two blocks per
// multiprocessor, into the caller's device image or into one of the two
// staging images copied on the copy stream; it releases the frame's pool when
// done. A frame whose composite was not launched gives its number back, so the
// pool's next march does not wait for a release that never comes.
vr_status composite_pipelined(vr_ctx ctx, vr_frame_s &fr, float *out, int out_on_device, cudaStream_t s,
                              const PoolSync &sync)
{
    const int blocks = ctx->sms > 0 ? 2 * ctx->sms : 0;
    vr_status st = VR_OK;
    if (out_on_device) {
        st = composite(ctx, fr, reinterpret_cast<float4 *>(out), s, blocks, &sync);
        if (st != VR_OK) ctx->pool_frame = sync.frame - 1;
        return st;
    }
    const long long px = static_cast<long long>(fr.W) * fr.H;
    float4 *buf = nullptr;
    int slot = -1;
    st = host_staging(ctx, px, s, &buf, &slot);
    if (st == VR_OK) st = composite(ctx, fr, buf, s, blocks, &sync);
    if (st != VR_OK) {
        ctx->pool_frame = sync.frame - 1;
        return st;
    }
    return host_copy(ctx, out, buf, slot, px, s);
}

// Ray-state cycling frame straight into the image (device or host output).
vr_status cycle_to(vr_ctx ctx, vr_volume vol, float *out, int out_on_device, cudaStream_t s)
{
    if (!out) return fail(ctx, VR_ERR_ARG, "null output");
    static thread_local MarchParams mp;
    vr_status st = prepare_frame(ctx, vol, ctx->frame, mp);
    if (st != VR_OK) return st;
    const long long px = static_cast<long long>(mp.W) * mp.H;
    float4 *dst = reinterpret_cast<float4 *>(out);
    int slot = -1;
    if (!out_on_device) {
        st = host_staging(ctx, px, s, &dst, &slot);
        if (st != VR_OK) return st;
    }
    // pipelined frames (see render_to): this frame's kernel may start in the
    // previous frame's tail; it reads only the bricks and the table before it
    // waits, and writes its image after the preceding grid completes
    const bool pipe = pipelined_output(ctx, out_on_device);
    const bool after = pipe_after(ctx, s) && pipe;
    const int t = timing_begin(ctx, 0, s);
    VR_LAUNCH(ctx, launch_march_cycle(mp, vol->kind(), dst, s, after));
    timing_end(ctx, t, s);
    if (!out_on_device) {
        st = host_copy(ctx, out, dst, slot, px, s);
        if (st != VR_OK) return st;
    }
    if (pipe) pipe_launched(ctx, s);
    return VR_OK;
}

// A sort-last frame into the caller's image. Pipelined frames (device output
// or asynchronous host output, kernel timing off, the quad march) alternate
// between the context's two frames and composite with a persistent grid of two
// blocks per multiprocessor, which is resident early in the march's tail; its
// blocks signal at their start,
// so the next frame's march (launched as a programmatic dependent when nothing
// it reads before its waits has changed, on the same stream) can fill the
// multiprocessors as this frame's march drains. Every write of that march waits
// for this composite's completion, and the pool it writes was last read by the
// frame before, whose composite precedes this one in the stream.
vr_status render_to(vr_ctx ctx, vr_volume vol, float *out, int out_on_device, cudaStream_t s)
{
    if (!out) return fail(ctx, VR_ERR_ARG, "null output");
    const bool pipe = pipelined_output(ctx, out_on_device) && !(ctx->staging && vol->d_scalar);
    if (!pipe) {
        ctx->pipe_ready = false;
        vr_status st = march(ctx, vol, ctx->frame, s);
        if (st != VR_OK) return st;
        return composite_to(ctx, ctx->frame, out, out_on_device, s);
    }
    const PoolSync sync = pipe_frame(ctx);
    vr_frame_s &fr = pipe_pool(ctx, sync);
    vr_status st = march(ctx, vol, fr, s, pipe_after(ctx, s), &sync);
    if (st != VR_OK) {
        ctx->pool_frame = sync.frame - 1;
        return st;
    }
    st = composite_pipelined(ctx, fr, out, out_on_device, s, sync);
    if (st != VR_OK) return st;
    pipe_launched(ctx, s);
    return VR_OK;
}

}  // namespace host
}  // namespace vr

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *vr_status_string(vr_status s)
{
    switch (s) {
    case VR_OK: return "ok";
    case VR_ERR_ARG: return "invalid argument";
    case VR_ERR_OOM: return "out of memory";
    case VR_ERR_CUDA: return "CUDA error";
    case VR_ERR_STATE: return "invalid state";
    case VR_ERR_TIMEOUT: return "device wait timed out";
    case VR_ERR_BOUNDS: return "device index check failed";
    }
    return "unknown status";
}

const char *vr_last_error(vr_ctx ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

vr_status vr_partition_boxes(const int dims[3], const vr_partition *part, int *n_bricks, int *boxes)
{
    std::vector<int> bx;
    std::vector<KdNode> tree;
    const char *why = nullptr;
    if (!partition_plan(dims, part, bx, tree, &why)) return VR_ERR_ARG;
    if (n_bricks) *n_bricks = static_cast<int>(bx.size() / 6);
    if (boxes) std::memcpy(boxes, bx.data(), bx.size() * sizeof(int));
    return VR_OK;
}

vr_status vr_plan_view(const int dims[3], const vr_partition *part, const vr_camera *cam, int *order, int *rects)
{
    std::vector<int> bx;
    std::vector<KdNode> tree;
    const char *why = nullptr;
    if (!partition_plan(dims, part, bx, tree, &why) || !camera_valid(cam)) return VR_ERR_ARG;
    Basis B;
    make_basis(*cam, B);
    const double nmax = nmax3(dims);
    const int nb = static_cast<int>(bx.size() / 6);
    if (order) {
        std::vector<int> o;
        visibility_order(tree, 0, *cam, nmax, o);
        std::memcpy(order, o.data(), o.size() * sizeof(int));
    }
    if (rects)
        for (int b = 0; b < nb; ++b) footprint(*cam, B, &bx[6 * b], nmax, rects + 4 * b);
    return VR_OK;
}

vr_status vr_create(int cuda_device, vr_ctx *out)
{
    if (!out) return VR_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || cuda_device < 0 || cuda_device >= n) {
        cudaGetLastError();
        return VR_ERR_ARG;
    }
    vr_ctx ctx = new (std::nothrow) vr_ctx_s;
    if (!ctx) return VR_ERR_OOM;
    ctx->device = cuda_device;
    DeviceGuard g(cuda_device);
    if (!g.ok || vr::host::dev_malloc(&ctx->d_counter, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(ctx->d_counter, 0, sizeof(unsigned long long)) != cudaSuccess ||
        vr::host::dev_malloc(&ctx->d_error, sizeof(int)) != cudaSuccess || cudaMemset(ctx->d_error, 0, sizeof(int)) != cudaSuccess ||
        vr::host::dev_malloc(&ctx->d_pool_done, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(ctx->d_pool_done, 0, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        vr::host::dev_malloc(&ctx->d_pool_count, 2 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(ctx->d_pool_count, 0, 2 * sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctx->d_counter);
        cudaFree(ctx->d_error);
        cudaFree(ctx->d_pool_done);
        cudaFree(ctx->d_pool_count);
        delete ctx;
        return VR_ERR_CUDA;
    }
    ctx->frame.owned_by_ctx = true;
    ctx->frame2.owned_by_ctx = true;
    if (cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, cuda_device) != cudaSuccess) {
        cudaGetLastError();
        ctx->sms = 0;
    }
    *out = ctx;
    return VR_OK;
}

vr_status vr_destroy(vr_ctx ctx)
{
    if (!ctx) return VR_ERR_ARG;
    if (ctx->live_objects != 0) return fail(ctx, VR_ERR_STATE, "volumes or frames still alive");
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    cudaFree(ctx->d_tf);
    cudaFree(ctx->d_counter);
    cudaFree(ctx->d_error);
    cudaFree(ctx->d_gpart);
    cudaFree(ctx->frame.d_part);
    cudaFree(ctx->frame2.d_part);
    cudaFree(ctx->d_pool_done);
    cudaFree(ctx->d_pool_count);
    cudaFree(ctx->d_img);
    if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
    for (int i = 0; i < 2; ++i) {
        cudaFree(ctx->d_img2[i]);
        if (ctx->ev_rendered[i]) cudaEventDestroy(ctx->ev_rendered[i]);
        if (ctx->ev_copied[i]) cudaEventDestroy(ctx->ev_copied[i]);
    }
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (auto &t : ctx->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    delete ctx;
    return VR_OK;
}

vr_status vr_set_kernel_timing(vr_ctx ctx, int on)
{
    if (!ctx) return VR_ERR_ARG;
    ctx->timing = on != 0;
    return VR_OK;
}

vr_status vr_get_kernel_timing(vr_ctx ctx, double *march_ms, long long *march_launches, double *composite_ms,
                               long long *composite_launches)
{
    if (!ctx) return VR_ERR_ARG;
    DeviceGuard g(ctx->device);
    double ms[2] = {0, 0};
    long long n[2] = {0, 0};
    vr_status st = VR_OK;
    for (auto &t : ctx->timed) {
        float e = 0.f;
        if (cudaEventSynchronize(t.b) == cudaSuccess && cudaEventElapsedTime(&e, t.a, t.b) == cudaSuccess) {
            ms[t.kind] += e;
            n[t.kind] += 1;
        } else {
            cudaGetLastError();
            st = fail(ctx, VR_ERR_CUDA, "kernel timing event failed");
        }
        ctx->event_pool.push_back(t.a);
        ctx->event_pool.push_back(t.b);
    }
    ctx->timed.clear();
    if (march_ms) *march_ms = ms[0];
    if (march_launches) *march_launches = n[0];
    if (composite_ms) *composite_ms = ms[1];
    if (composite_launches) *composite_launches = n[1];
    return st;
}

vr_status vr_sync(vr_ctx ctx, void *stream)
{
    if (!ctx) return VR_ERR_ARG;
    DeviceGuard g(ctx->device);
    VR_CUDA(ctx, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    if (ctx->copy_stream) VR_CUDA(ctx, cudaStreamSynchronize(ctx->copy_stream));
    int err = 0;
    VR_CUDA(ctx, cudaMemcpy(&err, ctx->d_error, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        VR_CUDA(ctx, cudaMemset(ctx->d_error, 0, sizeof(int)));
        if (err & 64) {
            // a pool wait gave up: once the device is idle, mark every pool as
            // released up to the current frame, so later frames do not wait
            VR_CUDA(ctx, cudaDeviceSynchronize());
            const unsigned long long done[2] = {ctx->pool_frame, ctx->pool_frame};
            VR_CUDA(ctx, cudaMemcpy(ctx->d_pool_done, done, sizeof(done), cudaMemcpyHostToDevice));
            VR_CUDA(ctx, cudaMemset(ctx->d_pool_count, 0, 2 * sizeof(unsigned int)));
            ctx->pipe_ready = false;
        }
        if (err & 2) return fail(ctx, VR_ERR_TIMEOUT, "a bounded device-side wait of the batched kernel gave up");
        if (err & 32) return fail(ctx, VR_ERR_TIMEOUT, "a bounded wait for a staged brick slab gave up");
        if (err & 64) return fail(ctx, VR_ERR_TIMEOUT, "a pipelined frame's bounded wait for its partial pool gave up");
        if (err & 8) return fail(ctx, VR_ERR_BOUNDS, "a mesh point location found no element");
        if (err & 16)
            return fail(ctx, VR_ERR_BOUNDS, "a counted sample's cell fell outside its brick's storage or staged box");
        return fail(ctx, VR_ERR_BOUNDS, "a backward pass met an owned-sample run longer than 4096 samples");
    }
    return VR_OK;
}

namespace {
vr_status create_volume(vr_ctx ctx, const int dims[3], vr_dtype storage, const vr_partition *part, int n_held,
                        const int *held, const float *src, int src_on_device, void *stream, vr_volume *out)
{
    if (!ctx || !out) return VR_ERR_ARG;
    *out = nullptr;
    if (!dims || !part || !src) return fail(ctx, VR_ERR_ARG, "null argument");
    if (storage != VR_F32 && storage != VR_BF16 && storage != VR_F16)
        return fail(ctx, VR_ERR_ARG, "unknown storage type");
    std::unique_ptr<vr_volume_s> vol(new (std::nothrow) vr_volume_s);
    if (!vol) return VR_ERR_OOM;
    vol->ctx = ctx;
    std::memcpy(vol->dims, dims, sizeof(vol->dims));
    vol->dtype = storage;
    vol->octets = storage != VR_F32 && ctx->cell_layout == 1;
    const char *why = nullptr;
    if (!partition_plan(dims, part, vol->boxes, vol->tree, &why)) return fail(ctx, VR_ERR_ARG, why);
    const int nb = static_cast<int>(vol->boxes.size() / 6);
    // quad indices inside a brick are 32-bit
    for (int b = 0; b < nb; ++b)
        if (brick_quads(&vol->boxes[6 * b]) > 0x7fffffffLL)
            return fail(ctx, VR_ERR_ARG, "a brick holds more than 2^31 - 1 quads (about 1290^3 voxels); use more bricks");
    if (held) {
        if (n_held < 1 || n_held > nb) return fail(ctx, VR_ERR_ARG, "a share holds 1 to n_bricks bricks");
        vol->held.assign(nb, 0);
        for (int i = 0; i < n_held; ++i) {
            if (held[i] < 0 || held[i] >= nb || vol->held[held[i]])
                return fail(ctx, VR_ERR_ARG, "share brick ids must be distinct brick ids of the partition");
            vol->held[held[i]] = 1;
        }
    }

    // brick-major haloed xy-quad (or octet) storage of the held bricks, each 256-byte aligned
    const size_t es = quad_size(storage, vol->octets);
    long long off_bytes = 0;
    vol->base.resize(nb);
    for (int b = 0; b < nb; ++b) {
        vol->base[b] = off_bytes / static_cast<long long>(es);
        if (!vol->holds(b)) continue;
        off_bytes += brick_quads(&vol->boxes[6 * b]) * static_cast<long long>(es);
        off_bytes = (off_bytes + 255) & ~255LL;
    }
    off_bytes = std::max(off_bytes, 256LL);
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    VR_CUDA(ctx, vr::host::dev_malloc(&vol->d_data, static_cast<size_t>(off_bytes)));
    vol->bytes = off_bytes;
    if (ctx->staging && storage == VR_F32) {
        // scalar copy for the staged march: rows padded to 4 elements (16 bytes),
        // each brick 128-byte aligned
        long long off = 0;
        vol->sbase.resize(nb);
        vol->sxp.resize(nb);
        for (int b = 0; b < nb; ++b) {
            const int *bx = &vol->boxes[6 * b];
            vol->sxp[b] = (bx[3] - bx[0] + 2 + 3) & ~3;
            vol->sbase[b] = off;
            if (!vol->holds(b)) continue;
            off += static_cast<long long>(vol->sxp[b]) * (bx[4] - bx[1] + 2) * (bx[5] - bx[2] + 2);
            off = (off + 31) & ~31LL;
        }
        off = std::max(off, 32LL);
        const cudaError_t es2 = vr::host::dev_malloc(&vol->d_scalar, static_cast<size_t>(off) * sizeof(float));
        if (es2 != cudaSuccess) {
            cudaFree(vol->d_data);
            return cuda_fail(ctx, es2, "scalar brick copy");
        }
        vol->bytes += off * static_cast<long long>(sizeof(float));
    }
    const float *dsrc = src;
    float *tmp = nullptr;
    const size_t nvox = static_cast<size_t>(dims[0]) * dims[1] * dims[2];
    if (!src_on_device) {
        cudaError_t e = vr::host::dev_malloc(&tmp, nvox * sizeof(float));
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, src, nvox * sizeof(float), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            cudaFree(vol->d_data);
            cudaFree(vol->d_scalar);
            return cuda_fail(ctx, e, "volume upload");
        }
        dsrc = tmp;
    }
    cudaError_t e = pack_bricks(vol.get(), dsrc, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) {
        cudaFree(vol->d_data);
        cudaFree(vol->d_scalar);
        return cuda_fail(ctx, e, "volume pack");
    }
    ctx->live_objects++;
    *out = vol.release();
    return VR_OK;
}
}  // namespace

vr_status vr_volume_create(vr_ctx ctx, const int dims[3], vr_dtype storage, const vr_partition *part,
                           const float *src, int src_on_device, void *stream, vr_volume *out)
{
    vr::host::TraceRange trace_("vr_volume_create");
    return create_volume(ctx, dims, storage, part, 0, nullptr, src, src_on_device, stream, out);
}

vr_status vr_volume_create_share(vr_ctx ctx, const int dims[3], vr_dtype storage, const vr_partition *part,
                                 int n_held, const int *held, const float *src, int src_on_device, void *stream,
                                 vr_volume *out)
{
    vr::host::TraceRange trace_("vr_volume_create_share");
    if (!held) return ctx ? fail(ctx, VR_ERR_ARG, "null share") : VR_ERR_ARG;
    return create_volume(ctx, dims, storage, part, n_held, held, src, src_on_device, stream, out);
}

vr_status vr_volume_update(vr_volume vol, const float *src, int src_on_device, void *stream)
{
    vr::host::TraceRange trace_("vr_volume_update");
    if (!vol || !src) return VR_ERR_ARG;
    vr_ctx ctx = vol->ctx;
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nvox = static_cast<size_t>(vol->dims[0]) * vol->dims[1] * vol->dims[2];
    const float *dsrc = src;
    float *tmp = nullptr;
    if (!src_on_device) {
        VR_CUDA(ctx, vr::host::dev_malloc(&tmp, nvox * sizeof(float)));
        cudaError_t e = cudaMemcpyAsync(tmp, src, nvox * sizeof(float), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cuda_fail(ctx, e, "volume upload");
        }
        dsrc = tmp;
    }
    cudaError_t e = pack_bricks(vol, dsrc, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "volume pack");
    return VR_OK;
}

vr_status vr_volume_update_async(vr_volume vol, const float *src, int src_on_device, void *stream)
{
    vr::host::TraceRange trace_("vr_volume_update_async");
    if (!vol || !src) return VR_ERR_ARG;
    vr_ctx ctx = vol->ctx;
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nvox = static_cast<size_t>(vol->dims[0]) * vol->dims[1] * vol->dims[2];
    const float *dsrc = src;
    if (!src_on_device) {
        if (!vol->d_staging) VR_CUDA(ctx, vr::host::dev_malloc(&vol->d_staging, nvox * sizeof(float)));
        VR_CUDA(ctx, cudaMemcpyAsync(vol->d_staging, src, nvox * sizeof(float), cudaMemcpyHostToDevice, s));
        dsrc = vol->d_staging;
    }
    VR_CUDA(ctx, pack_bricks(vol, dsrc, s));
    return VR_OK;
}

vr_status vr_render_backward(vr_ctx ctx, vr_volume vol, const float *grad_rgba_dev, float *grad_tf_dev,
                             float *grad_density_dev, void *stream)
{
    vr::host::TraceRange trace_("vr_render_backward");
    if (!ctx || !vol) return VR_ERR_ARG;
    if (!grad_rgba_dev || !grad_tf_dev) return fail(ctx, VR_ERR_ARG, "null gradient buffer");
    if (vol->ctx != ctx) return fail(ctx, VR_ERR_ARG, "volume belongs to another context");
    if (ctx->ert_alpha < 1.0f) return fail(ctx, VR_ERR_ARG, "backward requires early termination off");
    if (ctx->opc_ref > 0.0f) return fail(ctx, VR_ERR_ARG, "backward requires opacity correction off");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    static thread_local MarchParams mp;
    vr_frame_s &fr = ctx->frame;
    // forward partials (recomputed: nothing per sample is kept from the forward call)
    vr_status st = prepare_frame(ctx, vol, fr, mp);
    if (st != VR_OK) return st;
    st = ensure_frame(ctx, fr, std::max(fr.pool_px, 1LL));
    if (st != VR_OK) return st;
    mp.partials = fr.d_part;
    mp.sample_counter = nullptr;
    VR_LAUNCH(ctx, launch_march(mp, vol->kind(), s));
    if (fr.total_px > ctx->gpart_cap) {
        cudaFree(ctx->d_gpart);
        ctx->d_gpart = nullptr;
        ctx->gpart_cap = 0;
        VR_CUDA(ctx, vr::host::dev_malloc(&ctx->d_gpart, static_cast<size_t>(fr.total_px) * sizeof(float4)));
        ctx->gpart_cap = fr.total_px;
    }
    static thread_local CompositeGradParams cg;
    std::memset(&cg, 0, sizeof(cg));
    cg.W = fr.W;
    cg.H = fr.H;
    cg.nb = fr.nb;
    for (int j = 0; j < fr.nb; ++j) cg.order[j] = fr.order[j];
    for (int b = 0; b < fr.nb; ++b) {
        std::memcpy(cg.rect[b], &fr.rects[4 * b], 4 * sizeof(int));
        cg.poff[b] = fr.poff[b];
    }
    cg.partials = fr.d_part;
    cg.grad_img = reinterpret_cast<const float4 *>(grad_rgba_dev);
    cg.grad_partials = ctx->d_gpart;
    VR_LAUNCH(ctx, launch_composite_grad(cg, s));
    GradArgs ga;
    ga.grad_partials = ctx->d_gpart;
    ga.grad_tf = grad_tf_dev;
    ga.grad_vol = grad_density_dev;
    for (int a = 0; a < 3; ++a) ga.N[a] = vol->dims[a];
    ga.error = ctx->d_error;
    VR_LAUNCH(ctx, launch_march_grad(mp, ga, vol->kind(), s));
    return VR_OK;
}

vr_status vr_volume_release(vr_volume vol)
{
    if (!vol) return VR_ERR_ARG;
    DeviceGuard g(vol->ctx->device);
    cudaFree(vol->d_data);
    cudaFree(vol->d_staging);
    cudaFree(vol->d_scalar);
    vol->ctx->live_objects--;
    delete vol;
    return VR_OK;
}

vr_status vr_volume_info(vr_volume vol, int *n_bricks, int *boxes, long long *storage_bytes)
{
    if (!vol) return VR_ERR_ARG;
    if (n_bricks) *n_bricks = static_cast<int>(vol->boxes.size() / 6);
    if (boxes) std::memcpy(boxes, vol->boxes.data(), vol->boxes.size() * sizeof(int));
    if (storage_bytes) *storage_bytes = vol->bytes;
    return VR_OK;
}

vr_status vr_volume_read_brick(vr_volume vol, int brick, void *dst, size_t bytes)
{
    if (!vol || !dst) return VR_ERR_ARG;
    const int nb = static_cast<int>(vol->boxes.size() / 6);
    if (brick < 0 || brick >= nb) return fail(vol->ctx, VR_ERR_ARG, "brick index out of range");
    if (!vol->holds(brick)) return fail(vol->ctx, VR_ERR_ARG, "the brick is not in this volume's share");
    const int *bx = &vol->boxes[6 * brick];
    const int sx = bx[3] - bx[0] + 2, sy = bx[4] - bx[1] + 2, sz = bx[5] - bx[2] + 2;
    const size_t es = elem_size(vol->dtype);
    const size_t n = static_cast<size_t>(sx) * sy * sz * es;
    if (bytes < n) return fail(vol->ctx, VR_ERR_ARG, "destination too small");
    const long long nq = brick_quads(bx);
    const size_t per = vol->octets ? 8 : 4;  // voxels per storage element
    std::vector<unsigned char> q(static_cast<size_t>(nq) * per * es);
    DeviceGuard g(vol->ctx->device);
    VR_CUDA(vol->ctx, cudaMemcpy(q.data(), static_cast<const char *>(vol->d_data) +
                                               vol->base[brick] * static_cast<long long>(per * es),
                                 q.size(), cudaMemcpyDeviceToHost));
    // voxel (i,j,k) is component (i==sx-1) + 2*(j==sy-1) of quad (min(i,sx-2), min(j,sy-2), k);
    // with octets, quad k is the first half of element k, or for the last plane
    // the second half of element k-1
    const int qx = sx - 1, qy = sy - 1, nbx = sx / 2, nby = sy / 2;
    unsigned char *out = static_cast<unsigned char *>(dst);
    for (int k = 0; k < sz; ++k)
        for (int j = 0; j < sy; ++j)
            for (int i = 0; i < sx; ++i) {
                const int ii = std::min(i, qx - 1), jj = std::min(j, qy - 1);
                const int c = (i == sx - 1 ? 1 : 0) + (j == sy - 1 ? 2 : 0);
                const bool upper = vol->octets && k == sz - 1;
                const int kk = upper ? k - 1 : k;
                const size_t src = static_cast<size_t>(quad_index(ii, jj, kk, nbx, nby)) * per + (upper ? 4 : 0) + c;
                const size_t o = (static_cast<size_t>(k) * sy + j) * sx + i;
                std::memcpy(out + o * es, q.data() + src * es, es);
            }
    return VR_OK;
}

vr_status vr_set_transfer_function(vr_ctx ctx, const float *rgba, int n, float vmin, float vmax, int on_device)
{
    if (!ctx) return VR_ERR_ARG;
    if (!rgba || n < 2 || n > 1024 || !(vmax > vmin) || !std::isfinite(vmin) || !std::isfinite(vmax))
        return fail(ctx, VR_ERR_ARG, "bad transfer function");
    DeviceGuard g(ctx->device);
    if (n > ctx->tf_cap) {
        cudaFree(ctx->d_tf);
        ctx->d_tf = nullptr;
        ctx->tf_cap = 0;
        ctx->has_tf = false;
        VR_CUDA(ctx, vr::host::dev_malloc(&ctx->d_tf, 2 * static_cast<size_t>(n) * sizeof(float4)));
        ctx->tf_cap = n;
    }
    // device table: (T[i], T[i+1] - T[i]) pairs in float32, last difference 0
    std::vector<float> t(4 * static_cast<size_t>(n)), pairs(8 * static_cast<size_t>(n));
    if (on_device)
        VR_CUDA(ctx, cudaMemcpy(t.data(), rgba, t.size() * sizeof(float), cudaMemcpyDeviceToHost));
    else
        std::memcpy(t.data(), rgba, t.size() * sizeof(float));
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < 4; ++c) {
            const float a = t[4 * i + c];
            const float b = i + 1 < n ? t[4 * (i + 1) + c] : a;
            pairs[8 * i + c] = a;
            pairs[8 * i + 4 + c] = b - a;
        }
    ctx->input_seq++;  // a pipelined march must not read the table across this upload
    VR_CUDA(ctx, cudaMemcpy(ctx->d_tf, pairs.data(), pairs.size() * sizeof(float), cudaMemcpyHostToDevice));
    ctx->ntf = n;
    ctx->vmin = vmin;
    ctx->vmax = vmax;
    ctx->has_tf = true;
    return VR_OK;
}

vr_status vr_set_camera(vr_ctx ctx, const vr_camera *cam)
{
    if (!ctx) return VR_ERR_ARG;
    if (!camera_valid(cam)) return fail(ctx, VR_ERR_ARG, "bad camera (size, extent, field of view or basis)");
    ctx->cam = *cam;
    ctx->has_cam = true;
    return VR_OK;
}

vr_status vr_set_render_params(vr_ctx ctx, float step_voxels, float ert_alpha)
{
    if (!ctx) return VR_ERR_ARG;
    if (!(step_voxels > 0.0f) || !(ert_alpha > 0.0f)) return fail(ctx, VR_ERR_ARG, "bad render params");
    ctx->step = step_voxels;
    ctx->ert_alpha = ert_alpha;
    return VR_OK;
}

vr_status vr_set_composite_schedule(vr_ctx ctx, int n_factors, const int *factors)
{
    if (!ctx) return VR_ERR_ARG;
    if (n_factors < 0 || n_factors > kMaxFactors || (n_factors > 0 && !factors))
        return fail(ctx, VR_ERR_ARG, "bad schedule");
    for (int i = 0; i < n_factors; ++i)
        if (factors[i] < 1) return fail(ctx, VR_ERR_ARG, "bad schedule factor");
    ctx->factors.assign(factors, factors + n_factors);
    return VR_OK;
}

vr_status vr_set_count_samples(vr_ctx ctx, int on)
{
    if (!ctx) return VR_ERR_ARG;
    ctx->count_samples = on != 0;
    return VR_OK;
}

vr_status vr_get_sample_count(vr_ctx ctx, long long *count)
{
    if (!ctx || !count) return VR_ERR_ARG;
    DeviceGuard g(ctx->device);
    unsigned long long v = 0;
    VR_CUDA(ctx, cudaDeviceSynchronize());
    VR_CUDA(ctx, cudaMemcpy(&v, ctx->d_counter, sizeof(v), cudaMemcpyDeviceToHost));
    VR_CUDA(ctx, cudaMemset(ctx->d_counter, 0, sizeof(v)));
    *count = static_cast<long long>(v);
    return VR_OK;
}

vr_status vr_render_partials(vr_ctx ctx, vr_volume vol, vr_frame *out, void *stream)
{
    vr::host::TraceRange trace_("vr_render_partials");
    if (!ctx || !vol || !out) return VR_ERR_ARG;
    *out = nullptr;
    if (vol->ctx != ctx) return fail(ctx, VR_ERR_ARG, "volume belongs to another context");
    std::unique_ptr<vr_frame_s> fr(new (std::nothrow) vr_frame_s);
    if (!fr) return VR_ERR_OOM;
    DeviceGuard g(ctx->device);
    vr_status st = march(ctx, vol, *fr, static_cast<cudaStream_t>(stream));
    if (st != VR_OK) {
        cudaFree(fr->d_part);
        return st;
    }
    ctx->live_objects++;
    *out = fr.release();
    return VR_OK;
}

vr_status vr_frame_info(vr_frame fr, int *n_bricks, int *rects, int *order)
{
    if (!fr) return VR_ERR_ARG;
    if (n_bricks) *n_bricks = fr->nb;
    if (rects) std::memcpy(rects, fr->rects.data(), fr->rects.size() * sizeof(int));
    if (order) std::memcpy(order, fr->order.data(), fr->order.size() * sizeof(int));
    return VR_OK;
}

vr_status vr_frame_partial(vr_frame fr, int brick, const float **dev_ptr)
{
    if (!fr || !dev_ptr || brick < 0 || brick >= fr->nb) return VR_ERR_ARG;
    *dev_ptr = reinterpret_cast<const float *>(fr->d_part + fr->poff[brick]);
    return VR_OK;
}

vr_status vr_composite(vr_ctx ctx, vr_frame fr, float *out_rgba, int out_on_device, void *stream)
{
    vr::host::TraceRange trace_("vr_composite");
    if (!ctx || !fr) return VR_ERR_ARG;
    if (fr->ctx != ctx) return fail(ctx, VR_ERR_ARG, "frame belongs to another context");
    DeviceGuard g(ctx->device);
    return composite_to(ctx, *fr, out_rgba, out_on_device, static_cast<cudaStream_t>(stream));
}

vr_status vr_frame_release(vr_frame fr)
{
    if (!fr || fr->owned_by_ctx) return VR_ERR_ARG;
    DeviceGuard g(fr->ctx->device);
    cudaFree(fr->d_part);
    fr->ctx->live_objects--;
    delete fr;
    return VR_OK;
}

vr_status vr_render_frame(vr_ctx ctx, vr_volume vol, float *out_rgba, int out_on_device, void *stream)
{
    vr::host::TraceRange trace_("vr_render_frame");
    if (!ctx || !vol) return VR_ERR_ARG;
    if (vol->ctx != ctx) return fail(ctx, VR_ERR_ARG, "volume belongs to another context");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (ctx->mode == 1) return cycle_to(ctx, vol, out_rgba, out_on_device, s);
    return render_to(ctx, vol, out_rgba, out_on_device, s);
}

vr_status vr_debug_pipeline_gap(vr_ctx ctx)
{
    if (!ctx) return VR_ERR_ARG;
    ctx->pool_frame += 2;
    return VR_OK;
}

vr_status vr_set_frame_pipelining(vr_ctx ctx, int on)
{
    if (!ctx) return VR_ERR_ARG;
    ctx->pipelining = on != 0;
    ctx->pipe_ready = false;
    return VR_OK;
}

vr_status vr_set_opacity_correction(vr_ctx ctx, float ref_step_voxels)
{
    if (!ctx) return VR_ERR_ARG;
    if (!(ref_step_voxels >= 0.0f) || !std::isfinite(ref_step_voxels))
        return fail(ctx, VR_ERR_ARG, "bad reference step");
    ctx->opc_ref = ref_step_voxels;
    return VR_OK;
}

vr_status vr_set_host_output_async(vr_ctx ctx, int on)
{
    if (!ctx) return VR_ERR_ARG;
    ctx->host_async = on != 0;
    return VR_OK;
}

vr_status vr_composite_images(vr_ctx ctx, int n, const float *const *images_dev, float *out_dev, long long pixels,
                              void *stream)
{
    vr::host::TraceRange trace_("vr_composite_images");
    if (!ctx) return VR_ERR_ARG;
    if (n < 1 || n > kMaxBricks || !images_dev || !out_dev || pixels < 0)
        return fail(ctx, VR_ERR_ARG, "1 to VR_MAX_BRICKS images, an output and a pixel count >= 0");
    static thread_local ImagesParams ip;
    for (int j = 0; j < n; ++j) {
        if (!images_dev[j] || (reinterpret_cast<uintptr_t>(images_dev[j]) & 15))
            return fail(ctx, VR_ERR_ARG, "image pointers must be non-null and 16-byte aligned");
        ip.img[j] = reinterpret_cast<const float4 *>(images_dev[j]);
    }
    if (reinterpret_cast<uintptr_t>(out_dev) & 15) return fail(ctx, VR_ERR_ARG, "output must be 16-byte aligned");
    ip.n = n;
    ip.pixels = pixels;
    ip.out = reinterpret_cast<float4 *>(out_dev);
    DeviceGuard g(ctx->device);
    VR_LAUNCH(ctx, launch_composite_images(ip, static_cast<cudaStream_t>(stream)));
    return VR_OK;
}

vr_status vr_set_cell_layout(vr_ctx ctx, int layout)
{
    if (!ctx) return VR_ERR_ARG;
    if (layout != 0 && layout != 1) return fail(ctx, VR_ERR_ARG, "cell layout 0 (xy-quads) or 1 (octets)");
    ctx->cell_layout = layout;
    return VR_OK;
}

vr_status vr_set_march_staging(vr_ctx ctx, int on)
{
    if (!ctx) return VR_ERR_ARG;
    ctx->staging = on != 0;
    return VR_OK;
}

vr_status vr_set_packet_width(vr_ctx ctx, int packet_width)
{
    if (!ctx) return VR_ERR_ARG;
    if (packet_width != 4 && packet_width != 8 && packet_width != 16)
        return fail(ctx, VR_ERR_ARG, "packet width must be 4, 8 or 16");
    ctx->packet_width = packet_width;
    return VR_OK;
}

vr_status vr_set_render_mode(vr_ctx ctx, int mode)
{
    if (!ctx) return VR_ERR_ARG;
    if (mode != 0 && mode != 1) return fail(ctx, VR_ERR_ARG, "render mode must be 0 or 1");
    ctx->mode = mode;
    return VR_OK;
}

}  // extern "C"

vr_status vr_debug_inject_fault(int kind, int after)
{
    if (kind < VR_FAULT_NONE || kind > VR_FAULT_LAUNCH || after < 0) return VR_ERR_ARG;
    g_fault_kind.store(VR_FAULT_NONE);
    g_fault_after.store(after);
    g_fault_kind.store(kind);
    return VR_OK;
}
