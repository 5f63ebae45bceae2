// nrm_tree_s.cu -- the binary32 (S) tree kernels and their entry points
// (instantiated here from nrm_tree.cuh).
#include "nrm_tree.cuh"

namespace nrm {

nrm_status run_single_x(nrm_ctx *c, const float *x, int64_t n, float p, float *out, cudaStream_t s, int64_t item_lo,
                        int64_t item_hi, const VecPlan *plan_in, int64_t stride, int variant) {
    return run_single<float>(c, x, n, p, out, s, item_lo, item_hi, plan_in, stride, variant);
}

nrm_status run_batch_x(nrm_ctx *c, const float *x, int64_t x_len, const int64_t *off, const int64_t *lens,
                       int64_t B, float p, const double *p_dev, float *out, int32_t *status, cudaStream_t s,
                       float *lanes) {
    return run_batch<float>(c, x, x_len, off, lens, B, p, p_dev, out, status, s, lanes);
}

} // namespace nrm
