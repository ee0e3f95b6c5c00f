// Sort-last distribution across ranks (Sections 2.3.1, 2.3.3 and 2.3.4 of
// arXiv:1205.0282):
//
//   kd_partition       Section 2.3.1: the cube is split into sub-cubes of (near)
//                      equal volume by a k-d tree over the bricks: each node cuts
//                      its longest axis, the two children taking shares of the
//                      node's ranks in proportion to their share of its bricks
//                      along that axis (a count that is not a power of two puts
//                      floor(n/2) ranks on the low side).
//   kd_order           visibility order of the k-d leaves from an eye point: the
//                      tree is walked with the eye's side of each cut first, so
//                      every ray meets the leaves it crosses in that order.
//   subimage_composite Sections 2.3.3-2.3.4: the root folds the ranks' rectangle-
//                      clipped sub-images front to back with 'over', stopping once
//                      a pixel is opaque.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "vr_internal.cuh"

namespace vr {

namespace {

struct KdNode {
    int32_t lo[3], hi[3];  // brick range [lo, hi)
    int32_t parts;         // ranks in this subtree
    int32_t axis, cut;     // inner node: cut plane at brick index `cut` along `axis`
    int32_t child[2];      // inner node children (-1 for a leaf)
    int32_t leaf;          // leaf number (tree order), -1 for inner nodes
};

// Voxel extent of the brick range [lo, hi) along axis a (its sampling region).
double extent(const int64_t n[3], const int32_t B[3], const int32_t lo[3], const int32_t hi[3], int a) {
    const double x0 = (double)lo[a] * B[a];
    const double x1 = std::min((double)hi[a] * B[a], (double)(n[a] - 1));
    return x1 - x0;
}

// Build the tree; returns false if some node must split a range of one brick.
bool build_tree(const int64_t n[3], const int32_t B[3], const int32_t nb[3], int32_t parts,
                std::vector<KdNode>& nodes) {
    nodes.clear();
    KdNode root{};
    for (int a = 0; a < 3; ++a) {
        root.lo[a] = 0;
        root.hi[a] = nb[a];
    }
    root.parts = parts;
    root.child[0] = root.child[1] = -1;
    root.leaf = -1;
    nodes.push_back(root);
    int32_t leaves = 0;
    // depth-first, low child first, so that leaves are numbered in tree order
    std::vector<int32_t> stack{0};
    while (!stack.empty()) {
        const int32_t id = stack.back();
        stack.pop_back();
        KdNode nd = nodes[id];
        if (nd.parts == 1) {
            nodes[id].leaf = leaves++;
            continue;
        }
        // longest axis by voxel extent that still has two bricks (ties: lowest axis)
        int ax = -1;
        double best = -1.0;
        for (int a = 0; a < 3; ++a) {
            if (nd.hi[a] - nd.lo[a] < 2) continue;
            const double e = extent(n, B, nd.lo, nd.hi, a);
            if (e > best) {
                best = e;
                ax = a;
            }
        }
        if (ax < 0) return false;
        const int32_t p0 = nd.parts / 2, p1 = nd.parts - p0;
        const int32_t len = nd.hi[ax] - nd.lo[ax];
        int32_t k = (int32_t)std::lround((double)len * p0 / nd.parts);
        k = std::min(std::max(k, 1), len - 1);
        nd.axis = ax;
        nd.cut = nd.lo[ax] + k;
        KdNode lo_child = nd, hi_child = nd;
        lo_child.hi[ax] = nd.cut;
        lo_child.parts = p0;
        hi_child.lo[ax] = nd.cut;
        hi_child.parts = p1;
        for (KdNode* ch : {&lo_child, &hi_child}) {
            ch->child[0] = ch->child[1] = -1;
            ch->leaf = -1;
        }
        nodes[id].axis = nd.axis;
        nodes[id].cut = nd.cut;
        nodes[id].child[0] = (int32_t)nodes.size();
        nodes.push_back(lo_child);
        nodes[id].child[1] = (int32_t)nodes.size();
        nodes.push_back(hi_child);
        stack.push_back(nodes[id].child[1]);
        stack.push_back(nodes[id].child[0]);
    }
    return true;
}

}  // namespace

bool kd_partition(const int64_t n[3], const int32_t B[3], int32_t parts, int32_t* ranges) {
    int32_t nb[3];
    for (int a = 0; a < 3; ++a) nb[a] = (int32_t)((n[a] - 1 + B[a] - 1) / B[a]);
    std::vector<KdNode> nodes;
    if (!build_tree(n, B, nb, parts, nodes)) return false;
    for (const KdNode& nd : nodes)
        if (nd.leaf >= 0)
            for (int a = 0; a < 3; ++a) {
                ranges[6 * nd.leaf + a] = nd.lo[a];
                ranges[6 * nd.leaf + 3 + a] = nd.hi[a];
            }
    return true;
}

bool kd_order(const int64_t n[3], const int32_t B[3], int32_t parts, const double eye[3], int32_t* order) {
    int32_t nb[3];
    for (int a = 0; a < 3; ++a) nb[a] = (int32_t)((n[a] - 1 + B[a] - 1) / B[a]);
    std::vector<KdNode> nodes;
    if (!build_tree(n, B, nb, parts, nodes)) return false;
    int32_t k = 0;
    std::vector<int32_t> stack{0};
    while (!stack.empty()) {
        const KdNode& nd = nodes[stack.back()];
        stack.pop_back();
        if (nd.leaf >= 0) {
            order[k++] = nd.leaf;
            continue;
        }
        // the cut plane in voxel coordinates; the eye's side is visited first
        const double plane = (double)nd.cut * B[nd.axis];
        const int first = eye[nd.axis] < plane ? 0 : 1;
        stack.push_back(nd.child[1 - first]);
        stack.push_back(nd.child[first]);
    }
    return k == parts;
}

// One thread per output pixel: fold the sub-images whose rectangle holds the
// pixel, in the listed (front-to-back) order, until the pixel is opaque.
__global__ void __launch_bounds__(256) subimage_composite_kernel(const SubimageList L, int32_t width,
                                                                  int32_t height, float tau,
                                                                  float4* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)width * height) return;
    const int i = (int)(idx % width), j = (int)(idx / width);
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int k = 0; k < L.n; ++k) {
        const SubimageRef& s = L.s[k];
        if (i < s.x0 || i > s.x1 || j < s.y0 || j > s.y1) continue;
        if (acc.w >= tau) break;
        const float4 fr = s.data[(int64_t)(j - s.y0) * (s.x1 - s.x0 + 1) + (i - s.x0)];
        const float tr = 1.0f - acc.w;
        acc.x = fmaf(tr, fr.x, acc.x);
        acc.y = fmaf(tr, fr.y, acc.y);
        acc.z = fmaf(tr, fr.z, acc.z);
        acc.w = fmaf(tr, fr.w, acc.w);
    }
    out[idx] = acc;
}

cudaError_t launch_subimage_composite(const SubimageList& L, int32_t width, int32_t height, float tau,
                                      float4* out, cudaStream_t s) {
    const int64_t px = (int64_t)width * height;
    subimage_composite_kernel<<<(unsigned)((px + 255) / 256), 256, 0, s>>>(L, width, height, tau, out);
    return cudaGetLastError();
}

}  // namespace vr
