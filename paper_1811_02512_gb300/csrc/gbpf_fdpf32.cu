// gbpf_fdpf32.cu -- the FP32 instantiations of the power-flow iteration
// kernels (gbpf_fdpf.cuh), compiled apart from the other precision's.
#include "gbpf_fdpf.cuh"

namespace gbpf {

cudaError_t fdpf_pack_f32(const RunArgs *args_dev, const int *order_dev, int ngrid, unsigned *counter_dev,
                          size_t smem, int blocks, cudaStream_t s) {
    return fdpf_pack_t<float>(args_dev, order_dev, ngrid, counter_dev, smem, blocks, s);
}

bool fdpf_clusters_fit_f32(int C, int ncase, size_t smem) { return fdpf_clusters_fit_t<float>(C, ncase, smem); }

cudaError_t fdpf_run_f32(const RunArgs &a, size_t smem, int cluster, int threads, cudaStream_t s) {
    return fdpf_run_t<float>(a, smem, cluster, threads, s);
}

}  // namespace gbpf
