// gbpf_fdpf.cu -- launchers of the power-flow iteration kernels
// (gbpf_fdpf.cuh; the kernels themselves are instantiated per precision in
// gbpf_fdpf64.cu and gbpf_fdpf32.cu).
#include "gbpf_fdpf.cuh"

namespace gbpf {

// ------------------------------------------------------------ launchers

cudaError_t launch_fdpf_pack(const RunArgs *args_dev, const int *order_dev, int ngrid,
                             unsigned *counter_dev, int prec, size_t smem, int nsm, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter_dev, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const int blocks = ngrid < nsm ? ngrid : nsm;
    return prec == PF_FP64 ? fdpf_pack_f64(args_dev, order_dev, ngrid, counter_dev, smem, blocks, s)
                           : fdpf_pack_f32(args_dev, order_dev, ngrid, counter_dev, smem, blocks, s);
}

// Fills the run arguments of one grid of a pack (the single-case form of
// launch_fdpf's arguments); use_smem is decided by the caller.
void fill_run_args(RunArgs &a, const DevNet &dn, const DevCases &dc, const DevMat *m, const void *F0,
                   const void *F1, const void *TV0, const void *TV1, const double *A0,
                   const double *A1, const int *fstat0, const int *fstat1, const pf_run_opts &o,
                   double *vm, double *va, double *ef, double *iv, double *xg, double *bmax,
                   pf_case_result *res) {
    a.TV0 = m[0].npf2 > 0 ? TV0 : nullptr;
    a.TV1 = m[1].npf2 > 0 ? TV1 : nullptr;
    a.TW0 = a.TW1 = nullptr;
    a.Z0 = a.Z1 = nullptr;
    a.K0 = a.K1 = nullptr;
    a.iv = iv;
    a.A0 = A0;
    a.A1 = A1;
    a.ir_max = o.ir_max;
    a.ir_tol = o.ir_tol;
    a.ir_abs = o.ir_abs > 0 ? o.ir_abs : 0.01 * o.tol;
    a.dn = dn;
    a.dc = dc;
    a.m0 = m[0];
    a.m1 = m[1];
    a.F0 = F0;
    a.F1 = F1;
    a.fs0 = fstat0;
    a.fs1 = fstat1;
    a.tol = o.tol;
    a.max_iter = o.max_iter;
    a.flat = o.flat_start;
    a.spin = o.spin_limit > 0 ? unsigned(o.spin_limit) : kDefaultSpin;
    a.vm = vm;
    a.va = va;
    a.ef = ef;
    a.xg = xg;
    a.bmax = bmax;
    a.res = res;
    a.use_smem = 0;
    a.fallback = 0;
}

size_t run_args_bytes() { return sizeof(RunArgs); }

cudaError_t launch_pack(const PackGrid *grids, int ngrid, int prec, const pf_run_opts &o,
                        const int *order_host, void *args_dev, int *order_dev, unsigned *counter_dev,
                        size_t smem_optin, int nsm, cudaStream_t s) {
    // the launch reserves shared memory for the largest grid whose solve
    // vector fits; larger grids keep theirs in global scratch
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    const size_t ring = size_t(kStages) * kStageBytes;
    int ns = 0;
    for (int g = 0; g < ngrid; g++) {
        const int nm = grids[g].m[0].n > grids[g].m[1].n ? grids[g].m[0].n : grids[g].m[1].n;
        if (ring + elt * size_t(nm) + 2048 <= smem_optin && nm > ns) ns = nm;
    }
    std::vector<RunArgs> A(static_cast<size_t>(ngrid));
    for (int g = 0; g < ngrid; g++) {
        const PackGrid &p = grids[g];
        fill_run_args(A[g], p.dn, p.dc, p.m, p.F0, p.F1, p.TV0, p.TV1, p.A0, p.A1, p.fs0, p.fs1, o,
                      p.vm, p.va, p.ef, p.iv, p.xg, p.bmax, p.res);
        const int nm = p.m[0].n > p.m[1].n ? p.m[0].n : p.m[1].n;
        A[g].use_smem = nm <= ns;
    }
    cudaError_t e = cudaMemcpyAsync(args_dev, A.data(), sizeof(RunArgs) * size_t(ngrid),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(order_dev, order_host, sizeof(int) * size_t(ngrid), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // A is released on return
    if (e != cudaSuccess) return e;
    return launch_fdpf_pack(static_cast<const RunArgs *>(args_dev), order_dev, ngrid, counter_dev, prec,
                            ring + elt * size_t(ns), nsm, s);
}

// Cluster size of the power-flow kernel: a case spreads its nodal work over
// 16 (or 8) SMs when the batch is too small to fill the GPU with one block per
// case and such clusters can be resident; otherwise one block per case.
int fdpf_cluster_size(int ncase, int num_sms, int prec, size_t smem_optin, int nmax) {
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    size_t smem = size_t(kStages) * kStageBytes + elt * size_t(nmax);
    if (smem + 2048 > smem_optin) smem = size_t(kStages) * kStageBytes;
    for (int C : {16, 8}) {
        if (ncase * C > num_sms) continue;
        if (prec == PF_FP64 ? fdpf_clusters_fit_f64(C, ncase, smem) : fdpf_clusters_fit_f32(C, ncase, smem))
            return C;
    }
    return 1;
}

cudaError_t launch_fdpf(const DevNet &dn, const DevCases &dc, const DevMat *m, int prec,
                        const void *F0, const void *F1, const void *TV0, const void *TV1,
                        const double *A0, const double *A1, const int *fstat0, const int *fstat1,
                        const pf_run_opts &o, double *vm, double *va, double *ef, double *iv,
                        double *xg, double *bmax, pf_case_result *res, size_t smem_optin,
                        size_t smem_per_sm, int cluster, int threads, cudaStream_t s, const void *Z0,
                        const void *Z1, const double *K0, const double *K1, const NrLaunch *fb,
                        const void *TW0, const void *TW1) {
    RunArgs a;
    a.Z0 = Z0;
    a.Z1 = Z1;
    a.K0 = K0;
    a.K1 = K1;
    a.TV0 = m[0].npf2 > 0 ? TV0 : nullptr;
    a.TV1 = m[1].npf2 > 0 ? TV1 : nullptr;
    a.TW0 = m[0].npf3 > 0 && a.TV0 ? TW0 : nullptr;
    a.TW1 = m[1].npf3 > 0 && a.TV1 ? TW1 : nullptr;
    a.iv = iv;
    a.A0 = A0;
    a.A1 = A1;
    a.ir_max = o.ir_max;
    a.ir_tol = o.ir_tol;
    a.ir_abs = o.ir_abs > 0 ? o.ir_abs : 0.01 * o.tol;
    a.dn = dn;
    a.dc = dc;
    a.m0 = m[0];
    a.m1 = m[1];
    a.F0 = F0;
    a.F1 = F1;
    a.fs0 = fstat0;
    a.fs1 = fstat1;
    a.tol = o.tol;
    a.max_iter = o.max_iter;
    a.flat = o.flat_start;
    a.spin = o.spin_limit > 0 ? unsigned(o.spin_limit) : kDefaultSpin;
    a.vm = vm;
    a.va = va;
    a.ef = ef;
    a.xg = xg;
    a.bmax = bmax;
    a.res = res;
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    const int nmax = m[0].n > m[1].n ? m[0].n : m[1].n;
    const size_t ring = size_t(kStages) * kStageBytes;
    size_t smem = ring + elt * size_t(nmax);
    a.use_smem = smem + 2048 <= smem_optin;
    // one block per case with fewer threads: as many blocks per SM as the
    // registers allow (64 per thread), the solve vector in shared memory
    // only when it does not lower that count
    if (cluster > 1 || (threads != 256 && threads != 128)) threads = kRunThreads;
    if (threads < kRunThreads) {
        const size_t blocks = size_t(65536 / (threads * 64)) < size_t(2048 / threads)
                                  ? size_t(65536 / (threads * 64)) : size_t(2048 / threads);
        const size_t budget = smem_per_sm / blocks;
        a.use_smem = smem + 2048 <= budget && smem + 2048 <= smem_optin;
    }
    if (!a.use_smem) smem = ring;
    a.fallback = 0;
    if (fb) {  // the Newton-Raphson fallback's factor scratch, when it fits
        const size_t need = nr_args_within(*fb, smem, a.nr);
        if (need + 2048 <= smem_optin) {
            smem = need;
            a.fallback = 1;
        }
    }
    return prec == PF_FP64 ? fdpf_run_f64(a, smem, cluster, threads, s)
                           : fdpf_run_f32(a, smem, cluster, threads, s);
}

}  // namespace gbpf
