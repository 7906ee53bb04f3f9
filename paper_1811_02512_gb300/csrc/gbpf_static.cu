// gbpf_static.cu -- allocation-free variant of the nodal P/Q mismatch.
//
// Some callers cannot allocate device memory at the point where they need a
// mismatch: processes that reserve their whole device budget at start-up
// and forbid any later allocation (real-time energy-management front ends
// with a fixed memory plan), or host applications whose own allocator owns
// all GPU memory.  pf_mismatch_static serves them: it takes every input and
// output as caller-owned device memory and keeps its only intermediate (the
// rectangular voltages e + jf) in a fixed file-scope device array, so the
// call itself never allocates or frees anything.
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "gbpf.h"

namespace {

// Rectangular voltages of one case: e in [0, PF_STATIC_MAX_BUS), f after it.
// 2 MiB, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_static_ef[2 * PF_STATIC_MAX_BUS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_static_ptr[kMaxDevices] = {nullptr};

// Device address of g_static_ef on the current device, looked up once per
// device.  Host code must not use the symbol itself: on the host it names a
// stand-in, not device memory.
cudaError_t static_scratch(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_ef);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

__global__ void k_static_rect(int nbus, const double *vm, const double *va, double *ef) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbus; i += gridDim.x * blockDim.x) {
        double s, c;
        sincos(va[i], &s, &c);
        ef[i] = vm[i] * c;
        ef[PF_STATIC_MAX_BUS + i] = vm[i] * s;
    }
}

__global__ void k_static_rows(int nbus, const int32_t *rowptr, const int32_t *col, const double *G,
                              const double *B, const int32_t *btype, const double *psp,
                              const double *qsp, const double *ef, double *dp, double *dq,
                              double *maxmis) {
    const double *e = ef;
    const double *f = ef + PF_STATIC_MAX_BUS;
    double mx = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbus; i += gridDim.x * blockDim.x) {
        double ir = 0.0, ii = 0.0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            const int k = col[p];
            ir += G[p] * e[k] - B[p] * f[k];
            ii += G[p] * f[k] + B[p] * e[k];
        }
        const double P = e[i] * ir + f[i] * ii;
        const double Q = f[i] * ir - e[i] * ii;
        const int t = btype[i];
        const double a = (t != PF_BUS_SLACK) ? psp[i] - P : 0.0;
        const double b = (t == PF_BUS_PQ) ? qsp[i] - Q : 0.0;
        dp[i] = a;
        dq[i] = b;
        double l = fmax(fabs(a), fabs(b));
        if (a != a || b != b) l = __longlong_as_double(0x7ff8000000000000ll);
        mx = (l > mx || l != l) ? l : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = (w > mx || w != w) ? w : mx;
    }
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned long long *>(maxmis),
                  static_cast<unsigned long long>(__double_as_longlong(mx)));
}

}  // namespace

extern "C" pf_status pf_mismatch_static(int32_t nbus, const int32_t *rowptr_dev,
                                        const int32_t *col_dev, const double *G_dev,
                                        const double *B_dev, const int32_t *btype_dev,
                                        const double *psp_dev, const double *qsp_dev,
                                        const double *vm_dev, const double *va_dev,
                                        double *dp_dev, double *dq_dev, double *maxmis_dev,
                                        void *stream) {
    if (nbus < 1 || nbus > PF_STATIC_MAX_BUS) return PF_ERR_ARG;
    if (!rowptr_dev || !col_dev || !G_dev || !B_dev || !btype_dev || !psp_dev || !qsp_dev ||
        !vm_dev || !va_dev || !dp_dev || !dq_dev || !maxmis_dev)
        return PF_ERR_ARG;
    double *ef = nullptr;
    if (static_scratch(&ef) != cudaSuccess) return PF_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the maximum is accumulated with atomics, so it must start at zero
    if (cudaMemsetAsync(maxmis_dev, 0, sizeof(double), s) != cudaSuccess) return PF_ERR_CUDA;
    const int threads = 256;
    const int blocks = (nbus + threads - 1) / threads;
    k_static_rect<<<blocks, threads, 0, s>>>(nbus, vm_dev, va_dev, ef);
    k_static_rows<<<blocks, threads, 0, s>>>(nbus, rowptr_dev, col_dev, G_dev, B_dev, btype_dev,
                                             psp_dev, qsp_dev, ef, dp_dev, dq_dev, maxmis_dev);
    return cudaGetLastError() == cudaSuccess ? PF_OK : PF_ERR_CUDA;
}
