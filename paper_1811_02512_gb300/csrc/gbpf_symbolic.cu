// gbpf_symbolic.cu -- elimination tree and level sets on the GPU (Section
// II.B of arxiv 1811.02512: FormEliminationTree, the leaf-peeling partition
// of Table I), for sm_103a.
//
// From the filled pattern of L the parent of column j is the smallest row
// below j in its column (a min-reduction over the column); the level of a
// node is 1 for a leaf and 1 + the largest level of its children otherwise,
// which is the same number as the round in which leaf peeling removes it.
// The levels are found in one bottom-up pass without barriers: every leaf
// starts a walk towards the root, each node records its level, raises its
// parent's largest child level and counts itself off the parent's children;
// the child that counts off last continues the walk with the parent.  Every
// walk only moves up and every node is passed on once, so the pass does
// O(n) work and waits on nothing.

#include <cstdint>

#include "gbpf.h"

namespace {

__global__ void k_etree_parent(int n, const int64_t *Lp, const int32_t *Li, int32_t *parent,
                               int32_t *nchild, int32_t *pending, int32_t *maxchild) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        int p = n;
        for (int64_t q = Lp[j]; q < Lp[j + 1]; q++) {
            const int i = Li[q];
            if (i > j && i < p) p = i;
        }
        parent[j] = p < n ? p : -1;
        nchild[j] = 0;
        pending[j] = 0;
        maxchild[j] = 0;
    }
}

__global__ void k_count_children(int n, const int32_t *parent, int32_t *nchild, int32_t *pending) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int p = parent[j];
        if (p >= 0) {
            atomicAdd(nchild + p, 1);
            atomicAdd(pending + p, 1);
        }
    }
}

__global__ void k_levels(int n, const int32_t *parent, const int32_t *nchild, int32_t *pending,
                         int32_t *maxchild, int32_t *level, int32_t *nlev) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        if (nchild[j] != 0) continue;  // walks start at the leaves
        int node = j, lvl = 1;
        for (;;) {
            level[node] = lvl;
            const int p = parent[node];
            if (p < 0) {
                atomicMax(nlev, lvl);
                break;
            }
            atomicMax(maxchild + p, lvl);
            __threadfence();
            if (atomicSub(pending + p, 1) != 1) break;  // a sibling is still on its way
            __threadfence();
            lvl = atomicAdd(maxchild + p, 0) + 1;       // every child has raised it by now
            node = p;
        }
    }
}

}  // namespace

extern "C" pf_status pf_etree_levels_device(int32_t n, const int64_t *Lp_dev, const int32_t *Li_dev,
                                            int32_t *parent_dev, int32_t *level_dev, int32_t *nlev_dev,
                                            int32_t *scratch_dev, void *stream) {
    if (n < 1 || !Lp_dev || !Li_dev || !parent_dev || !level_dev || !nlev_dev || !scratch_dev)
        return PF_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t *nchild = scratch_dev, *pending = scratch_dev + n, *maxchild = scratch_dev + 2 * size_t(n);
    int blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (cudaMemsetAsync(nlev_dev, 0, sizeof(int32_t), s) != cudaSuccess) return PF_ERR_CUDA;
    k_etree_parent<<<blocks, 256, 0, s>>>(n, Lp_dev, Li_dev, parent_dev, nchild, pending, maxchild);
    k_count_children<<<blocks, 256, 0, s>>>(n, parent_dev, nchild, pending);
    k_levels<<<blocks, 256, 0, s>>>(n, parent_dev, nchild, pending, maxchild, level_dev, nlev_dev);
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_ERR_CUDA;
}
