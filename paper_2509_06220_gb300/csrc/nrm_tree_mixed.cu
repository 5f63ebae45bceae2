// nrm_tree_mixed.cu -- the persistent batch kernel with one p per vector
// (tree_kernel_mixed of nrm_tree.cuh), both element types.
#include "nrm_tree.cuh"

namespace nrm {

cudaError_t launch_mixed(nrm_ctx *c, const TreeArgs<double> &a, int64_t grid_warps, cudaStream_t s) {
    return launch_tree_mixed<double>(c, a, grid_warps, s);
}

cudaError_t launch_mixed(nrm_ctx *c, const TreeArgs<float> &a, int64_t grid_warps, cudaStream_t s) {
    return launch_tree_mixed<float>(c, a, grid_warps, s);
}

} // namespace nrm
