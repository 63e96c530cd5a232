// vr_mesh.h -- structures shared by the host runtime of tetrahedral-mesh volumes
// (vr_mesh_host.cpp) and their march kernel (vr_mesh.cu). Not part of the
// public ABI.
//
// The paper's data set is a mixed finite-element mesh distributed over ranks
// (Sec. 5); elements here are tetrahedra, each held by one brick. Within an
// element the value is linear, so along a ray it is linear in t, and a ray
// leaves the element through the face whose barycentric coordinate reaches 0
// first. A ray's run inside a brick therefore starts with one point location
// (a per-brick BVH, the acceleration structure of Sec. 2.1) and then walks
// face neighbours.
#pragma once

#include "vr_internal.h"

namespace vr {

// Element record, 4 float4 (64 B), voxel units:
//   r0 = (c.x, c.y, c.z, s_mean)   centroid and mean vertex value
//   ri = (n_i.x, n_i.y, n_i.z, s_i - s_0), i = 1..3
// with n_i the gradient of barycentric coordinate lambda_i, so that
// lambda_i(q) = 1/4 + n_i . (q - c) for i = 1..3, n_0 = -(n_1 + n_2 + n_3),
// and value(q) = s_mean + g . (q - c), g = sum_{i=1..3} (s_i - s_0) n_i.
// Face i is the face opposite vertex i (lambda_i = 0 on it).
constexpr int kMeshRec = 4;

// BVH node over a brick's elements (voxel units), nodes in preorder: an inner
// node's first child is the next node; `skip` is the first node after the
// node's subtree (the root's skip is the node count), so a point query needs no
// stack. leaf = 0 for an inner node, else (count << 28) | first: count elements
// from brick-local element index first.
struct MeshNode {
    float lo[3];
    int skip;
    float hi[3];
    int leaf;
};

constexpr int kMeshLeafMax = 4;        // elements per leaf
constexpr int kMeshMaxElems = 1 << 28; // elements per brick (leaf encoding)
constexpr int kMeshStallSteps = 32;    // element steps without a sample before re-locating

struct MeshParams {
    MarchParams m;                    // camera, lattice, transfer function, tiles, bricks
    const float4 *rec;                // kMeshRec float4 per element
    const int4 *nbr;                  // brick-local neighbour across face i, -1 on the brick's boundary
    const MeshNode *nodes;
    long long rec_base[kMaxBricks];   // first element of each brick
    long long node_base[kMaxBricks];  // first BVH node of each brick
    int *error;                       // bit 3: a point location found no element (empty brick)
};

// The grid starts with p.m.mask_blocks blocks that write the composite's tile
// masks. after_frame: launch as a programmatic dependent of the preceding
// kernel (the previous pipelined frame).
cudaError_t launch_march_mesh(const MeshParams &p, cudaStream_t s, bool after_frame = false);

}  // namespace vr
