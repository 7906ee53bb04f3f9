// gbpf_nr.cu -- Newton-Raphson power flow (Section III of arxiv 1811.02512)
// and its adjoint, for sm_103a: the kernels and their launchers; the device
// code of one Newton-Raphson case is in gbpf_nr.cuh.
#include "gbpf_nr.cuh"

namespace gbpf {

namespace {

// Newton-Raphson power flow of one case per cluster of C CTAs (nr_case).
template <class T, int C>
__global__ void __launch_bounds__(512, C == 1 ? 2 : 1) k_nr(NrArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[33];
    __shared__ Ring R;
    ring_init(&R);
    nr_case<T, C>(a, int(blockIdx.x) / C, C == 1 ? 0 : int(cluster_rank()), smem_raw, red, &R);
}

// Adjoint of case c: J(x)^T y = g with the stored factors (from the last
// Newton step, i.e. of an earlier state) refined in FP64 against the exact
// J(x) assembled here; dJ/dP_i = y_P(i), dJ/dQ_i = y_Q(i) (PQ), 0 elsewhere.
template <class T, int C>
__global__ void __launch_bounds__(512, C == 1 ? 2 : 1) k_adjoint(NrArgs a, int factor_now) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[33];
    __shared__ Ring R;
    const DevNet &dn = a.dn;
    const DevMat &m = a.m;
    const int nbus = dn.nbus;
    const int c = blockIdx.x / C;
    const int rank = C == 1 ? 0 : int(cluster_rank());
    unsigned char *stages = smem_raw;
    unsigned char *scratch = smem_raw + kStages * kStageBytes;
    T *xs = a.use_smem ? reinterpret_cast<T *>(scratch) : nullptr;
    ring_init(&R);
    T *F = static_cast<T *>(a.F) + (long long)c * m.jstride;
    const double *A = a.A + (long long)c * m.jstride;
    const int slice = (nbus + C - 1) / C;
    const int i0 = rank * slice, i1 = min(nbus, i0 + slice);
    const int nslot = m.n + m.nnz;
    const int sslice = (nslot + C - 1) / C;
    const int s0 = rank * sslice, s1 = min(nslot, s0 + sslice);
    double *flag = a.bmax + (long long)c * 16 + 15;
    nr_rect(a, c, i0, i1);
    cluster_sync<C>();
    (void)nr_mismatch_slice(a, c, i0, i1, red);  // P, Q at the state
    double *b = a.xg + (long long)c * 6 * nbus;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int k = m.new_of_bus[i];
        if (k >= 0) {
            b[2 * k] = a.gva[(long long)c * nbus + i];
            b[2 * k + 1] = dn.btype[i] == PF_BUS_PQ ? a.gvm[(long long)c * nbus + i] : 0.0;
        }
    }
    cluster_sync<C>();
    nr_assemble(a, c, s0, s1);
    cluster_sync<C>();
    int fsn = PF_OK;
    if (factor_now) fsn = cluster_block_factor<T, C>(a, c, rank, F, A, scratch, red, a.epoch0 + 1u);
    if (rank == 0) {
        int fs = factor_now ? fsn : a.fstat[c];
        int irs = 0;
        bool ok = fs == PF_OK;
        if (ok) ok = nr_solve<T, true>(a, &R, stages, xs, F, A, c, red, irs, true);
        if (threadIdx.x == 0) *flag = fs != PF_OK ? double(fs) : (ok ? 0.0 : double(PF_ERR_TIMEOUT));
    }
    cluster_sync<C>();
    const double *y = a.xg + (long long)c * 6 * nbus + 2 * nbus;
    const bool okall = *flag == 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int k = m.new_of_bus[i];
        const long long idx = (long long)c * nbus + i;
        double p = 0.0, q = 0.0;
        if (k >= 0 && okall) {
            p = y[2 * k];
            q = dn.btype[i] == PF_BUS_PQ ? y[2 * k + 1] : 0.0;
        } else if (!okall) {
            p = q = __longlong_as_double(0x7ff8000000000000ll);
        }
        a.dJdP[idx] = p;
        a.dJdQ[idx] = q;
    }
    if (rank == 0 && threadIdx.x == 0) a.res[c].status = okall ? PF_OK : int(*flag);
    cluster_sync<C>();
}

// Objective J = sum_i (V_i - 1)^2 + sum_i P_i (total active losses) of case c
// (one block per case) and its gradient with respect to every bus angle and
// magnitude: dJ/dtheta_k = sum_l dP_l/dtheta_k, dJ/dV_k = 2 (V_k - 1) +
// sum_l dP_l/dV_k, summed over every row l including the slack.
__global__ void __launch_bounds__(512) k_objective(DevNet dn, DevCases dc, const double *vm,
                                                   const double *va, double *ef, double *Jv,
                                                   double *gva, double *gvm) {
    __shared__ double red[33];
    const int c = blockIdx.x;
    const int nbus = dn.nbus;
    const double *v = vm + (long long)c * nbus;
    const double *th = va + (long long)c * nbus;
    double *e = ef + (long long)c * 4 * nbus;
    double *f = e + nbus;
    double *P = e + 2 * nbus;
    double *Q = e + 3 * nbus;
    const int outage = dc.outage[c];
    for (int i = threadIdx.x; i < nbus; i += blockDim.x) {
        double s, co;
        sincos(th[i], &s, &co);
        e[i] = v[i] * co;
        f[i] = v[i] * s;
    }
    __syncthreads();
    double part = 0.0;
    for (int i = threadIdx.x; i < nbus; i += blockDim.x) {
        double p, q;
        bus_injection(dn, i, outage, e, f, p, q);
        P[i] = p;
        Q[i] = q;
        part += (v[i] - 1.0) * (v[i] - 1.0) + p;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nbus; k += blockDim.x) {
        double gt = 0.0, gv = 2.0 * (v[k] - 1.0);
        for (int p = dn.rowptr[k]; p < dn.rowptr[k + 1]; p++) {
            const int l = dn.col[p];
            double G, B;
            y_entry(dn, outage, l, k, p, G, B);  // Y is symmetric: Y_lk at row k's slot
            if (l != k) {
                const B2<double> J = jac_off(G, B, e[l], f[l], e[k], f[k], v[k], false, false);
                gt += J.a;
                gv += J.b;
            } else {
                const B2<double> J = jac_diag(G, B, P[k], Q[k], v[k], false);
                gt += J.a;
                gv += J.b;
            }
        }
        gva[(long long)c * nbus + k] = gt;
        gvm[(long long)c * nbus + k] = gv;
    }
    // block sum of the objective (fixed order: warp shuffles then warps)
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); w++) s += red[w];
        Jv[c] = s;
    }
}

template <int C, class... Args>
cudaError_t launch_cluster(void (*kernel)(Args...), size_t smem, cudaStream_t s, int ncase,
                           Args... args) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(ncase) * C);
    cfg.blockDim = dim3(512);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    cfg.numAttrs = 0;
    if (C > 1) {
        if (C > 8) {
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace

// ------------------------------------------------------------ launchers

// Update terms staged per warp by the block factor: the most (up to
// kNrChunkMax, at least 32) that fit beside the ring and the accumulators.
int nr_chunk(const DevMat &m, int prec, size_t smem_optin) {
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    const size_t ring = size_t(kStages) * kStageBytes;
    const size_t room = smem_optin > ring + 4096 ? smem_optin - ring - 4096 : 0;
    const long long per_warp = (long long)(room / (512 / 32) / elt) - 8LL * (m.max_col + 1);
    long long ch = per_warp / 8;
    if (ch > kNrChunkMax) ch = kNrChunkMax;
    if (ch < 32) ch = 32;
    return int(ch);
}

size_t nr_smem(const DevMat &m, int prec, size_t smem_optin, int *use_smem) {
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    const size_t ring = size_t(kStages) * kStageBytes;
    const size_t fac = elt * size_t(8 * (m.max_col + 1) + 8 * nr_chunk(m, prec, smem_optin)) * (512 / 32);
    const size_t vec = elt * size_t(2 * m.n);
    size_t smem = ring + (fac > vec ? fac : vec);
    *use_smem = smem + 2048 <= smem_optin;
    if (!*use_smem) smem = ring + fac;
    return smem;
}

int nr_cluster_size(const DevMat &m, int ncase, int num_sms, int prec, size_t smem_optin) {
    int use = 0;
    const size_t smem = nr_smem(m, prec, smem_optin, &use);
    for (int C : {16, 8}) {
        if (ncase * C > num_sms) continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(unsigned(C));
        cfg.blockDim = dim3(512);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        cudaError_t e;
        if (prec == PF_FP64) {
            auto *k = (C == 16) ? k_nr<double, 16> : k_nr<double, 8>;
            if (C == 16) cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            e = cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg);
        } else {
            auto *k = (C == 16) ? k_nr<float, 16> : k_nr<float, 8>;
            if (C == 16) cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            e = cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg);
        }
        if (e == cudaSuccess && nclusters >= ncase) return C;
        cudaGetLastError();
    }
    return 1;
}

namespace {
void fill_nr_args(const NrLaunch &L, NrArgs &a) {
    a.dn = L.dn;
    a.dc = L.dc;
    a.m = L.m;
    a.F = L.F;
    a.A = L.A;
    a.fstat = L.fstat;
    a.tol = L.o.tol;
    a.max_iter = L.o.max_iter;
    a.flat = L.o.flat_start;
    a.spin = L.o.spin_limit > 0 ? unsigned(L.o.spin_limit) : kDefaultSpin;
    a.ir_max = L.o.ir_max;
    a.ir_tol = L.o.ir_tol;
    a.ir_abs = L.o.ir_abs > 0 ? L.o.ir_abs : 0.01 * L.o.tol;
    a.vm = L.vm;
    a.va = L.va;
    a.ef = L.ef;
    a.xg = L.xg;
    a.bmax = L.bmax;
    a.res = L.res;
    a.gva = L.gva;
    a.gvm = L.gvm;
    a.dJdP = L.dJdP;
    a.dJdQ = L.dJdQ;
    a.jdone = L.jdone;
    a.jsync = L.jsync;
    a.epoch0 = L.epoch0;
}
}  // namespace

size_t nr_args_within(const NrLaunch &L, size_t smem, NrArgs &a) {
    fill_nr_args(L, a);
    const size_t elt = L.prec == PF_FP64 ? sizeof(double) : sizeof(float);
    const size_t ring = size_t(kStages) * kStageBytes;
    const size_t warps = 512 / 32;
    const size_t acc = elt * warps * 8 * size_t(L.m.max_col + 1);  // accumulators of every warp
    const size_t per_term = elt * warps * 8;                       // one staged term in every warp
    if (smem < ring + acc + 32 * per_term) smem = ring + acc + 32 * per_term;
    size_t ch = (smem - ring - acc) / per_term;
    if (ch > size_t(kNrChunkMax)) ch = kNrChunkMax;
    a.fchunk = int(ch);
    a.use_smem = ring + elt * 2 * size_t(L.m.n) <= smem;
    return smem;
}

cudaError_t launch_nr(const NrLaunch &L, cudaStream_t s) {
    NrArgs a;
    fill_nr_args(L, a);
    a.fchunk = nr_chunk(L.m, L.prec, L.smem_optin);
    int use = 0;
    const size_t smem = nr_smem(L.m, L.prec, L.smem_optin, &use);
    a.use_smem = use;
    const int C = L.cluster;
    const int nc = L.dc.ncase;
    const int fnow = L.factor_now;
    if (L.adjoint) {
        if (L.prec == PF_FP64) {
            if (C >= 16) return launch_cluster<16>(k_adjoint<double, 16>, smem, s, nc, a, fnow);
            if (C >= 8) return launch_cluster<8>(k_adjoint<double, 8>, smem, s, nc, a, fnow);
            return launch_cluster<1>(k_adjoint<double, 1>, smem, s, nc, a, fnow);
        }
        if (C >= 16) return launch_cluster<16>(k_adjoint<float, 16>, smem, s, nc, a, fnow);
        if (C >= 8) return launch_cluster<8>(k_adjoint<float, 8>, smem, s, nc, a, fnow);
        return launch_cluster<1>(k_adjoint<float, 1>, smem, s, nc, a, fnow);
    }
    if (L.prec == PF_FP64) {
        if (C >= 16) return launch_cluster<16>(k_nr<double, 16>, smem, s, nc, a);
        if (C >= 8) return launch_cluster<8>(k_nr<double, 8>, smem, s, nc, a);
        return launch_cluster<1>(k_nr<double, 1>, smem, s, nc, a);
    }
    if (C >= 16) return launch_cluster<16>(k_nr<float, 16>, smem, s, nc, a);
    if (C >= 8) return launch_cluster<8>(k_nr<float, 8>, smem, s, nc, a);
    return launch_cluster<1>(k_nr<float, 1>, smem, s, nc, a);
}

cudaError_t launch_objective(const DevNet &dn, const DevCases &dc, const double *vm, const double *va,
                             double *ef, double *J, double *gva, double *gvm, cudaStream_t s) {
    k_objective<<<dc.ncase, 512, 0, s>>>(dn, dc, vm, va, ef, J, gva, gvm);
    return cudaGetLastError();
}

}  // namespace gbpf
