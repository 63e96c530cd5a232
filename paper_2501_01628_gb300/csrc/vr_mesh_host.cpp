// vr_mesh_host.cpp -- host runtime of tetrahedral-mesh volumes: assignment of
// elements to bricks, per-brick BVH and face adjacency, element records, and the
// C ABI (vr_mesh_*, vr_render_mesh_frame).
//
// Sec. 5 of arXiv:2501.01628: the rendered data set is a mixed finite-element
// mesh kept in the distribution the simulation used (each rank holds whole
// elements, unevenly spread in space). Sec. 2.1: rays find the elements they
// meet through a bounding volume hierarchy. Elements here are tetrahedra.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "vr_mesh.h"
#include "vr_objects.h"

using namespace vr;
using namespace vr::host;

struct vr_mesh_s {
    vr_ctx ctx = nullptr;
    vr_volume_s geom;                  // dims, boxes, kd tree; no voxel storage
    float4 *d_rec = nullptr;
    int4 *d_nbr = nullptr;
    MeshNode *d_nodes = nullptr;
    std::vector<long long> rec_base;   // per brick
    std::vector<long long> node_base;
    std::vector<long long> count;
    long long bytes = 0;
};

namespace {

struct BrickBuild {
    std::vector<long long> elems;   // global element ids in BVH leaf order
    std::vector<MeshNode> nodes;
    std::vector<float4> rec;
    std::vector<int4> nbr;
    std::string err;
};

struct MeshInput {
    const float *verts;
    const float *vals;
    const int *tets;
    long long nv, nt;
    double nmax;
};

// Vertex j of element e in voxel units (double).
inline void vtx(const MeshInput &in, long long e, int j, double v[3])
{
    const long long i = in.tets[4 * e + j];
    for (int a = 0; a < 3; ++a) v[a] = static_cast<double>(in.verts[3 * i + a]) * in.nmax;
}

// Median-split BVH over the brick's elements (centroids along the longest axis
// of their bounds), nodes in preorder with skip links (see vr_mesh.h);
// reorders b.elems into leaf order.
struct BvhBuilder {
    std::vector<std::array<float, 9>> box;  // per element: lo xyz, hi xyz, centroid xyz
    std::vector<long long> idx;
    std::vector<MeshNode> *nodes;

    void build(long long begin, long long end)
    {
        const int me = static_cast<int>(nodes->size());
        nodes->push_back(MeshNode{});
        MeshNode nd{};
        float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int a = 0; a < 3; ++a) {
            nd.lo[a] = INFINITY;
            nd.hi[a] = -INFINITY;
        }
        for (long long i = begin; i < end; ++i) {
            const auto &bx = box[idx[i]];
            for (int a = 0; a < 3; ++a) {
                nd.lo[a] = std::min(nd.lo[a], bx[a]);
                nd.hi[a] = std::max(nd.hi[a], bx[3 + a]);
                clo[a] = std::min(clo[a], bx[6 + a]);
                chi[a] = std::max(chi[a], bx[6 + a]);
            }
        }
        const long long cnt = end - begin;
        if (cnt <= kMeshLeafMax) {
            nd.leaf = static_cast<int>((cnt << 28) | begin);
        } else {
            int axis = 0;
            for (int a = 1; a < 3; ++a)
                if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
            const long long mid = begin + cnt / 2;
            std::nth_element(idx.begin() + begin, idx.begin() + mid, idx.begin() + end,
                             [&](long long x, long long y) { return box[x][6 + axis] < box[y][6 + axis]; });
            build(begin, mid);  // depth log2(n / 4): recursion stays shallow
            build(mid, end);
            nd.leaf = 0;
        }
        nd.skip = static_cast<int>(nodes->size());
        (*nodes)[me] = nd;
    }
};

bool build_bvh(const MeshInput &in, BrickBuild &b)
{
    const long long n = static_cast<long long>(b.elems.size());
    if (n >= kMeshMaxElems) {
        b.err = "too many elements in one brick";
        return false;
    }
    BvhBuilder B;
    B.box.resize(n);
    for (long long i = 0; i < n; ++i) {
        auto &bx = B.box[i];
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, c[3] = {0, 0, 0};
        for (int j = 0; j < 4; ++j) {
            double v[3];
            vtx(in, b.elems[i], j, v);
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], v[a]);
                hi[a] = std::max(hi[a], v[a]);
                c[a] += 0.25 * v[a];
            }
        }
        for (int a = 0; a < 3; ++a) {
            bx[a] = std::nextafter(static_cast<float>(lo[a]), -INFINITY);
            bx[3 + a] = std::nextafter(static_cast<float>(hi[a]), INFINITY);
            bx[6 + a] = static_cast<float>(c[a]);
        }
    }
    B.idx.resize(n);
    for (long long i = 0; i < n; ++i) B.idx[i] = i;
    b.nodes.clear();
    b.nodes.reserve(static_cast<size_t>(2 * (n / 2 + 1)));
    B.nodes = &b.nodes;
    B.build(0, n);
    std::vector<long long> ordered(n);
    for (long long i = 0; i < n; ++i) ordered[i] = b.elems[B.idx[i]];
    b.elems.swap(ordered);
    return true;
}

// Records (see vr_mesh.h) and face neighbours of the brick's elements, in
// b.elems order, with validation against the brick's box.
bool build_records(const MeshInput &in, const int *box, BrickBuild &b)
{
    const long long n = static_cast<long long>(b.elems.size());
    b.rec.resize(static_cast<size_t>(kMeshRec) * n);
    b.nbr.resize(n);
    double vol_sum = 0.0;
    constexpr double tol = 1e-3;  // voxel units
    for (long long i = 0; i < n; ++i) {
        const long long e = b.elems[i];
        double v[4][3], s[4];
        for (int j = 0; j < 4; ++j) {
            vtx(in, e, j, v[j]);
            s[j] = in.vals[in.tets[4 * e + j]];
            for (int a = 0; a < 3; ++a)
                if (v[j][a] < box[a] - tol || v[j][a] > box[3 + a] + tol) {
                    b.err = "an element reaches outside the brick that holds its centroid";
                    return false;
                }
        }
        double M[3][3];  // columns v1-v0, v2-v0, v3-v0
        for (int a = 0; a < 3; ++a)
            for (int j = 0; j < 3; ++j) M[a][j] = v[j + 1][a] - v[0][a];
        const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                           M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                           M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
        double scale = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int j = 0; j < 3; ++j) scale = std::max(scale, std::fabs(M[a][j]));
        if (!(std::fabs(det) > 1e-9 * scale * scale * scale)) {
            b.err = "degenerate element";
            return false;
        }
        vol_sum += std::fabs(det) / 6.0;
        // inverse by the adjugate: row j of M^-1 is the gradient of lambda_{j+1}
        double inv[3][3];
        inv[0][0] = (M[1][1] * M[2][2] - M[1][2] * M[2][1]) / det;
        inv[0][1] = (M[0][2] * M[2][1] - M[0][1] * M[2][2]) / det;
        inv[0][2] = (M[0][1] * M[1][2] - M[0][2] * M[1][1]) / det;
        inv[1][0] = (M[1][2] * M[2][0] - M[1][0] * M[2][2]) / det;
        inv[1][1] = (M[0][0] * M[2][2] - M[0][2] * M[2][0]) / det;
        inv[1][2] = (M[0][2] * M[1][0] - M[0][0] * M[1][2]) / det;
        inv[2][0] = (M[1][0] * M[2][1] - M[1][1] * M[2][0]) / det;
        inv[2][1] = (M[0][1] * M[2][0] - M[0][0] * M[2][1]) / det;
        inv[2][2] = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) / det;
        float4 *r = &b.rec[static_cast<size_t>(kMeshRec) * i];
        double c[3];
        for (int a = 0; a < 3; ++a) c[a] = 0.25 * (v[0][a] + v[1][a] + v[2][a] + v[3][a]);
        r[0] = make_float4(static_cast<float>(c[0]), static_cast<float>(c[1]), static_cast<float>(c[2]),
                           static_cast<float>(0.25 * (s[0] + s[1] + s[2] + s[3])));
        for (int j = 0; j < 3; ++j)
            r[j + 1] = make_float4(static_cast<float>(inv[j][0]), static_cast<float>(inv[j][1]),
                                   static_cast<float>(inv[j][2]), static_cast<float>(s[j + 1] - s[0]));
    }
    const double box_vol = static_cast<double>(box[3] - box[0]) * (box[4] - box[1]) * (box[5] - box[2]);
    if (std::fabs(vol_sum - box_vol) > 1e-4 * box_vol) {
        b.err = "the elements of a brick do not fill its box (gap or overlap)";
        return false;
    }
    // face neighbours: equal sorted vertex triples
    struct Face {
        int v[3];
        long long code;  // local element * 4 + face
    };
    std::vector<Face> faces(4 * static_cast<size_t>(n));
    for (long long i = 0; i < n; ++i) {
        const int *t = in.tets + 4 * b.elems[i];
        for (int f = 0; f < 4; ++f) {
            Face &F = faces[4 * i + f];
            int k = 0;
            for (int j = 0; j < 4; ++j)
                if (j != f) F.v[k++] = t[j];
            std::sort(F.v, F.v + 3);
            F.code = 4 * i + f;
        }
        b.nbr[i] = make_int4(-1, -1, -1, -1);
    }
    std::sort(faces.begin(), faces.end(), [](const Face &x, const Face &y) {
        return std::lexicographical_compare(x.v, x.v + 3, y.v, y.v + 3);
    });
    auto same = [](const Face &x, const Face &y) { return x.v[0] == y.v[0] && x.v[1] == y.v[1] && x.v[2] == y.v[2]; };
    auto set = [&](long long code, int other) {
        int4 &q = b.nbr[code >> 2];
        switch (code & 3) {
        case 0: q.x = other; break;
        case 1: q.y = other; break;
        case 2: q.z = other; break;
        default: q.w = other; break;
        }
    };
    for (size_t i = 0; i < faces.size();) {
        size_t j = i + 1;
        while (j < faces.size() && same(faces[i], faces[j])) ++j;
        if (j - i > 2) {
            b.err = "a face is shared by more than two elements";
            return false;
        }
        if (j - i == 2) {
            set(faces[i].code, static_cast<int>(faces[i + 1].code >> 2));
            set(faces[i + 1].code, static_cast<int>(faces[i].code >> 2));
        }
        i = j;
    }
    return true;
}

}  // namespace

extern "C" {

vr_status vr_mesh_create(vr_ctx ctx, const int dims[3], const vr_partition *part, const float *verts,
                         long long n_verts, const float *values, const int *tets, long long n_tets, vr_mesh *out)
{
    vr::host::TraceRange trace_("vr_mesh_create");
    if (!ctx || !out) return VR_ERR_ARG;
    *out = nullptr;
    if (!dims || !part || !verts || !values || !tets) return fail(ctx, VR_ERR_ARG, "null argument");
    if (n_verts < 4 || n_tets < 1 || n_verts > (1LL << 31) - 1)
        return fail(ctx, VR_ERR_ARG, "a mesh needs 4..2^31-1 vertices and at least one element");
    std::unique_ptr<vr_mesh_s> m(new (std::nothrow) vr_mesh_s);
    if (!m) return VR_ERR_OOM;
    m->ctx = ctx;
    vr_volume_s &G = m->geom;
    G.ctx = ctx;
    std::memcpy(G.dims, dims, sizeof(G.dims));
    const char *why = nullptr;
    if (!partition_plan(dims, part, G.boxes, G.tree, &why)) return fail(ctx, VR_ERR_ARG, why);
    const int nb = static_cast<int>(G.boxes.size() / 6);
    G.base.assign(nb, 0);
    for (long long i = 0; i < 4 * n_tets; ++i)
        if (tets[i] < 0 || tets[i] >= n_verts) return fail(ctx, VR_ERR_ARG, "element vertex index out of range");
    const MeshInput in{verts, values, tets, n_verts, n_tets, static_cast<double>(nmax3(dims))};

    // element -> brick: the brick whose box holds the centroid's cell
    std::vector<BrickBuild> bricks(nb);
    {
        std::vector<int> owner(n_tets);
        std::vector<long long> cnt(nb, 0);
        for (long long e = 0; e < n_tets; ++e) {
            int c[3];
            for (int a = 0; a < 3; ++a) {
                double sum = 0.0;
                for (int j = 0; j < 4; ++j) sum += verts[3 * static_cast<long long>(tets[4 * e + j]) + a];
                const double cell = std::floor(sum * 0.25 * in.nmax);
                c[a] = static_cast<int>(std::min(std::max(cell, 0.0), static_cast<double>(dims[a] - 1)));
            }
            owner[e] = -1;
            for (int b = 0; b < nb; ++b) {
                const int *bx = &G.boxes[6 * b];
                if (c[0] >= bx[0] && c[0] < bx[3] && c[1] >= bx[1] && c[1] < bx[4] && c[2] >= bx[2] && c[2] < bx[5]) {
                    owner[e] = b;
                    break;
                }
            }
            if (owner[e] < 0) return fail(ctx, VR_ERR_ARG, "an element's centroid lies in no brick");
            cnt[owner[e]]++;
        }
        for (int b = 0; b < nb; ++b) {
            if (cnt[b] == 0) return fail(ctx, VR_ERR_ARG, "a brick holds no element");
            if (cnt[b] > (1LL << 31) - 1) return fail(ctx, VR_ERR_ARG, "too many elements in one brick");
            bricks[b].elems.reserve(cnt[b]);
        }
        for (long long e = 0; e < n_tets; ++e) bricks[owner[e]].elems.push_back(e);
    }
    // per-brick BVH, records and adjacency, bricks in parallel
    {
        const int nthreads = std::max(1, std::min<int>(nb, static_cast<int>(std::thread::hardware_concurrency())));
        std::vector<std::thread> pool;
        std::atomic<int> next{0};
        for (int t = 0; t < nthreads; ++t)
            pool.emplace_back([&]() {
                for (int b = next++; b < nb; b = next++)
                    if (build_bvh(in, bricks[b])) build_records(in, &G.boxes[6 * b], bricks[b]);
            });
        for (auto &th : pool) th.join();
        for (int b = 0; b < nb; ++b)
            if (!bricks[b].err.empty()) return fail(ctx, VR_ERR_ARG, bricks[b].err);
    }
    long long n_rec = 0, n_nodes = 0;
    m->rec_base.resize(nb);
    m->node_base.resize(nb);
    m->count.resize(nb);
    for (int b = 0; b < nb; ++b) {
        m->rec_base[b] = n_rec;
        m->node_base[b] = n_nodes;
        m->count[b] = static_cast<long long>(bricks[b].elems.size());
        n_rec += m->count[b];
        n_nodes += static_cast<long long>(bricks[b].nodes.size());
    }
    DeviceGuard g(ctx->device);
    const size_t rec_bytes = static_cast<size_t>(n_rec) * kMeshRec * sizeof(float4);
    const size_t nbr_bytes = static_cast<size_t>(n_rec) * sizeof(int4);
    const size_t node_bytes = static_cast<size_t>(n_nodes) * sizeof(MeshNode);
    auto release = [&]() {
        cudaFree(m->d_rec);
        cudaFree(m->d_nbr);
        cudaFree(m->d_nodes);
    };
    cudaError_t e = vr::host::dev_malloc(&m->d_rec, rec_bytes);
    if (e == cudaSuccess) e = vr::host::dev_malloc(&m->d_nbr, nbr_bytes);
    if (e == cudaSuccess) e = vr::host::dev_malloc(&m->d_nodes, node_bytes);
    for (int b = 0; e == cudaSuccess && b < nb; ++b) {
        const BrickBuild &B = bricks[b];
        e = cudaMemcpy(m->d_rec + kMeshRec * m->rec_base[b], B.rec.data(), B.rec.size() * sizeof(float4),
                       cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(m->d_nbr + m->rec_base[b], B.nbr.data(), B.nbr.size() * sizeof(int4),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(m->d_nodes + m->node_base[b], B.nodes.data(), B.nodes.size() * sizeof(MeshNode),
                           cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        release();
        return cuda_fail(ctx, e, "mesh upload");
    }
    m->bytes = static_cast<long long>(rec_bytes + nbr_bytes + node_bytes);
    ctx->live_objects++;
    ctx->input_seq++;  // new device data a pipelined kernel must not overlap
    *out = m.release();
    return VR_OK;
}

vr_status vr_mesh_release(vr_mesh mesh)
{
    if (!mesh) return VR_ERR_ARG;
    DeviceGuard g(mesh->ctx->device);
    cudaFree(mesh->d_rec);
    cudaFree(mesh->d_nbr);
    cudaFree(mesh->d_nodes);
    mesh->ctx->live_objects--;
    delete mesh;
    return VR_OK;
}

vr_status vr_mesh_info(vr_mesh mesh, int *n_bricks, long long *elements_per_brick, long long *device_bytes)
{
    if (!mesh) return VR_ERR_ARG;
    const int nb = static_cast<int>(mesh->count.size());
    if (n_bricks) *n_bricks = nb;
    if (elements_per_brick) std::copy(mesh->count.begin(), mesh->count.end(), elements_per_brick);
    if (device_bytes) *device_bytes = mesh->bytes;
    return VR_OK;
}

vr_status vr_render_mesh_frame(vr_ctx ctx, vr_mesh mesh, float *out_rgba, int out_on_device, void *stream)
{
    vr::host::TraceRange trace_("vr_render_mesh_frame");
    if (!ctx || !mesh) return VR_ERR_ARG;
    if (mesh->ctx != ctx) return fail(ctx, VR_ERR_ARG, "mesh belongs to another context");
    if (!out_rgba) return fail(ctx, VR_ERR_ARG, "null output");
    if (ctx->mode != 0) return fail(ctx, VR_ERR_STATE, "meshes render in the sort-last mode only");
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    static thread_local MeshParams mp;  // ~15 KB: keep off the stack
    // pipelined frames as for volumes (vr_set_frame_pipelining)
    const bool pipe = vr::host::pipelined_output(ctx, out_on_device);
    const bool after = vr::host::pipe_after(ctx, s) && pipe;
    PoolSync sync{};
    if (pipe) sync = vr::host::pipe_frame(ctx);
    vr_frame_s &fr = pipe ? vr::host::pipe_pool(ctx, sync) : ctx->frame;
    auto give_back = [&](vr_status e) {  // no composite will release this frame's pool
        if (pipe) ctx->pool_frame = sync.frame - 1;
        return e;
    };
    vr_status st = prepare_frame(ctx, &mesh->geom, fr, mp.m);
    if (st != VR_OK) return give_back(st);
    st = ensure_frame(ctx, fr, std::max(fr.pool_px, 1LL));
    if (st != VR_OK) return give_back(st);
    mp.m.partials = fr.d_part;
    if (pipe) {
        mp.m.pool_done = sync.done;
        mp.m.pool_frame = sync.frame;
        mp.m.pool = sync.pool;
    }
    // the grid's first blocks write the composite's tile masks
    mp.m.tile_mask = reinterpret_cast<uint4 *>(fr.d_part + fr.total_px);
    mp.m.mask_tiles_x = fr.tiles_x;
    mp.m.mask_tiles_y = fr.tiles_y;
    mp.m.mask_blocks = (fr.tiles_x * fr.tiles_y + kMaskThreads - 1) / kMaskThreads;
    mp.rec = mesh->d_rec;
    mp.nbr = mesh->d_nbr;
    mp.nodes = mesh->d_nodes;
    for (size_t b = 0; b < mesh->rec_base.size(); ++b) {
        mp.rec_base[b] = mesh->rec_base[b];
        mp.node_base[b] = mesh->node_base[b];
    }
    mp.error = ctx->d_error;
    const int t = timing_begin(ctx, 0, s);
    st = [&]() -> vr_status {
        VR_LAUNCH(ctx, launch_march_mesh(mp, s, after));
        return VR_OK;
    }();
    if (st != VR_OK) return give_back(st);
    timing_end(ctx, t, s);
    fr.masks_ready = true;
    if (!pipe) return composite_to(ctx, fr, out_rgba, out_on_device, s);
    st = vr::host::composite_pipelined(ctx, fr, out_rgba, out_on_device, s, sync);
    if (st != VR_OK) return st;
    vr::host::pipe_launched(ctx, s);
    return VR_OK;
}

}  // extern "C"
