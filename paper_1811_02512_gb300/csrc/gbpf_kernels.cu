// gbpf_kernels.cu -- device kernels of libgbpf for sm_103a (GB300).
//
// Mapping of the paper's two kinds of parallelism (arxiv 1811.02512):
//  * nodal parallelism (Section II.A): one thread per bus row for the
//    admittance matrix (Section III.A, FormMatrixA) and for the P/Q
//    injections and mismatch;
//  * hierarchical parallelism (Section II.B): the levels of the elimination
//    tree run in order, separated by a block barrier; the columns (rows) of
//    one level run in parallel -- one warp per column in the numeric factor
//    (Section III.B), one thread per row/column in the substitutions
//    (Section III.C).
// One thread block owns one factor instance or one power-flow case for the
// whole computation, so a batch of cases fills the GPU with independent
// blocks and needs no grid-wide synchronisation at all.
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "gbpf_internal.h"

namespace gbpf {

namespace {

constexpr int kFactorThreads = 512;
constexpr int kSolveThreads = 512;
constexpr int kRunThreads = 512;

__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) {
        double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = (w > v || w != w) ? w : v;  // NaN wins
    }
    return v;
}

// Block-wide maximum of v (NaN wins); every thread receives the result.
// `red` is a 33-entry shared array.  Contains two __syncthreads.
__device__ double block_max(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_max(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double w = (lane < int(blockDim.x >> 5)) ? red[lane] : 0.0;
        w = warp_max(w);
        if (lane == 0) red[32] = w;
    }
    __syncthreads();
    return red[32];
}

// Atomic maximum of a non-negative double through its bit pattern (IEEE order
// of non-negative doubles equals integer order; NaN patterns sort above Inf).
__device__ void atomic_max_nonneg(double *addr, double v) {
    unsigned long long bits = __double_as_longlong(v);
    atomicMax(reinterpret_cast<unsigned long long *>(addr), bits);
}

// ------------------------------------------------------------ Section III.A

// FormMatrixA: row i of Y = G + jB is owned by one thread, which sums the
// pi models of the in-service branches incident to bus i (ascending branch
// index) and the bus shunt.  Also writes the XB B' (1/x weights) on the same
// pattern.
__global__ void k_ybus(DevNet dn) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dn.nbus) return;
    for (int p = dn.rowptr[i]; p < dn.rowptr[i + 1]; p++) {
        dn.G[p] = 0.0;
        dn.B[p] = 0.0;
        dn.Bp[p] = 0.0;
    }
    double gd = 0.0, bd = 0.0, bpd = 0.0;
    for (int q = dn.inc_ptr[i]; q < dn.inc_ptr[i + 1]; q++) {
        const int e = dn.inc_br[q];
        if (!dn.bstatus[e]) continue;
        const double r = dn.br[e], x = dn.bx[e], b = dn.bb[e], t = dn.btap[e];
        const double den = r * r + x * x;
        const double ys_re = r / den, ys_im = -x / den;
        const int po = dn.inc_pos[q];
        dn.G[po] -= ys_re / t;
        dn.B[po] -= ys_im / t;
        dn.Bp[po] -= 1.0 / x;
        if (dn.inc_side[q] == 0) {
            gd += ys_re / (t * t);
            bd += (ys_im + 0.5 * b) / (t * t);
        } else {
            gd += ys_re;
            bd += ys_im + 0.5 * b;
        }
        bpd += 1.0 / x;
    }
    const int d = dn.ydiag[i];
    dn.G[d] = gd + dn.gs[i];
    dn.B[d] = bd + dn.bs[i];
    dn.Bp[d] = bpd;
}

// Specified injections of every case: P = pg - pd s, Q = -qd s with the load
// scale s of PQ buses.
__global__ void k_case_spec(DevNet dn, DevCases dc, const double *ls) {
    const long long total = (long long)dc.ncase * dn.nbus;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = int(idx % dn.nbus);
        const double s = (ls && dn.btype[i] == PF_BUS_PQ) ? ls[idx] : 1.0;
        dc.Psp[idx] = dn.pg[i] - __dmul_rn(dn.pd[i], s);
        dc.Qsp[idx] = -__dmul_rn(dn.qd[i], s);
    }
}

// Contribution of branch e to slot s of B' (which = 0) or B'' (which = 1),
// used to take an outaged branch out of an assembled matrix.
__device__ double branch_slot_value(const DevNet &dn, const DevMat &m, int which, int e, int s) {
    const int sf = m.br_slot[3 * e], st = m.br_slot[3 * e + 1], sl = m.br_slot[3 * e + 2];
    const double r = dn.br[e], x = dn.bx[e], b = dn.bb[e], t = dn.btap[e];
    if (which == PF_MAT_BP) {
        if (s == sf || s == st) return 1.0 / x;
        if (s == sl) return -1.0 / x;
        return 0.0;
    }
    const double ys_im = -x / (r * r + x * x);
    if (s == sf) return -(ys_im + 0.5 * b) / (t * t);
    if (s == st) return -(ys_im + 0.5 * b);
    if (s == sl) return ys_im / t;
    return 0.0;
}

// Values of B' or B'' of every factor instance in slot layout: n diagonal
// slots (step order) then the strict-lower slots of L (fill slots zero).
__global__ void k_assemble_slots(DevNet dn, DevCases dc, DevMat m, int which, double *A) {
    const int per = m.n + m.nnz_l;
    const long long total = (long long)dc.ninst * per;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int inst = int(idx / per), s = int(idx % per);
        const int src = m.src[s];
        double v = 0.0;
        if (src >= 0) v = (which == PF_MAT_BP) ? dn.Bp[src] : -dn.B[src];
        const int e = dc.inst_outage[inst];
        if (e >= 0 && dn.bstatus[e]) v -= branch_slot_value(dn, m, which, e, s);
        A[(long long)inst * m.stride + s] = v;
    }
}

// ------------------------------------------------------------ Section III.B

// Numeric factor A = L D L^T of one instance per block, left-looking, level by
// level (FactorizeGraphA).  Column j of a level is owned by one warp: it
// gathers the updates a_ij -= l_ik d_k l_jk from every descendant column k in
// row j of L (ascending k, so the order of operations is fixed), then
// normalises l_ij = a_ij / d_j.  Columns of one level never write the same
// entry, so no atomics are needed and results are deterministic.
template <class T>
__global__ void __launch_bounds__(kFactorThreads)
    k_factor_ldlt(DevMat m, const double *A, T *F, int *fstatus) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[33];
    __shared__ int bad;
    const int inst = blockIdx.x;
    const int n = m.n;
    const double *a = A + (long long)inst * m.stride;
    T *v = F + (long long)inst * m.stride;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    T *acc = reinterpret_cast<T *>(smem_raw) + warp * (m.max_col + 1);
    if (threadIdx.x == 0) bad = PF_OK;
    double amax = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) amax = fmax(amax, fabs(a[j]));
    amax = block_max(amax, red);  // its barriers also publish `bad`
    const double piv_tol = 1e-14 * amax;
    for (int lev = 0; lev < m.nlev; lev++) {
        const int c1 = m.lvl_ptr[lev + 1];
        for (int ci = m.lvl_ptr[lev] + warp; ci < c1; ci += nwarps) {
            const int j = m.lvl_cols[ci];
            const int c0 = m.Lp[j], cnt = m.Lp[j + 1] - c0;
            for (int t = lane; t <= cnt; t += 32) acc[t] = T(t == 0 ? a[j] : a[n + c0 + t - 1]);
            __syncwarp();
            for (int q = m.Rp[j]; q < m.Rp[j + 1]; q++) {
                const int k = m.Rk[q], pkj = m.Rpos[q];
                const T mult = v[n + pkj] * v[k];
                const int len = m.Lp[k + 1] - pkj, o = m.uoff[q];
                for (int t = lane; t < len; t += 32) acc[m.umap[o + t]] -= v[n + pkj + t] * mult;
                __syncwarp();
            }
            const T d = acc[0];
            if (lane == 0) {
                v[j] = d;
                const double dd = double(d);
                if (!isfinite(dd)) atomicCAS(&bad, PF_OK, PF_ERR_NONFINITE);
                else if (fabs(dd) <= piv_tol) atomicCAS(&bad, PF_OK, PF_ERR_SINGULAR);
            }
            for (int t = lane; t < cnt; t += 32) v[n + c0 + t] = acc[1 + t] / d;
            __syncwarp();
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) fstatus[inst] = bad;
}

// ------------------------------------------------------------ Section III.C

// Solves L D L^T x = x in place for one block: forward substitution
// z_i = b_i - sum_k l_ik z_k by levels ascending (row lists), normalisation
// y_i = z_i / d_i (Eq. 4), back substitution x_k = y_k - sum_i l_ik x_i by
// levels descending (columns).  x is in step order, shared or global memory.
template <class T, class X>
__device__ void block_solve(const DevMat &m, const T *__restrict__ v, X *x) {
    const int n = m.n;
    for (int lev = 0; lev < m.nlev; lev++) {
        const int c1 = m.lvl_ptr[lev + 1];
        for (int ci = m.lvl_ptr[lev] + threadIdx.x; ci < c1; ci += blockDim.x) {
            const int i = m.lvl_cols[ci];
            X s = x[i];
            for (int q = m.Rp[i]; q < m.Rp[i + 1]; q++) s -= X(v[n + m.Rpos[q]]) * x[m.Rk[q]];
            x[i] = s;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = x[i] / X(v[i]);
    __syncthreads();
    for (int lev = m.nlev - 1; lev >= 0; lev--) {
        const int c1 = m.lvl_ptr[lev + 1];
        for (int ci = m.lvl_ptr[lev] + threadIdx.x; ci < c1; ci += blockDim.x) {
            const int k = m.lvl_cols[ci];
            X s = x[k];
            for (int p = m.Lp[k]; p < m.Lp[k + 1]; p++) s -= X(v[n + p]) * x[m.Li[p]];
            x[k] = s;
        }
        __syncthreads();
    }
}

template <class T>
__global__ void __launch_bounds__(kSolveThreads)
    k_solve(DevMat m, const T *F, const int *inst_of_case, double *rhs, T *gvec, int use_smem) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = blockIdx.x;
    const int n = m.n;
    const T *v = F + (long long)inst_of_case[c] * m.stride;
    T *x = use_smem ? reinterpret_cast<T *>(smem_raw) : gvec + (long long)c * 2 * n;
    double *r = rhs + (long long)c * n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) x[k] = T(r[m.perm[k]]);
    __syncthreads();
    block_solve<T, T>(m, v, x);
    for (int k = threadIdx.x; k < n; k += blockDim.x) r[m.perm[k]] = double(x[k]);
}

// ------------------------------------------------------------ Section II.A

__global__ void k_polar_to_rect(int nbus, int ncase, const double *vm, const double *va,
                                double *ef) {
    const long long total = (long long)ncase * nbus;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long c = idx / nbus;
        const int i = int(idx % nbus);
        double s, co;
        sincos(va[idx], &s, &co);
        ef[c * 2 * nbus + i] = vm[idx] * co;
        ef[c * 2 * nbus + nbus + i] = vm[idx] * s;
    }
}

// Injection at bus i of one case: I_i = sum_k Y_ik V_k on the base admittance
// matrix, minus the terms of the case's outaged branch (if any) at its end
// buses; returns S_i = V_i conj(I_i) as (P, Q).
__device__ __forceinline__ void bus_injection(const DevNet &dn, int i, int outage,
                                              const double *e, const double *f, double &P,
                                              double &Q) {
    double ir = 0.0, ii = 0.0;
    for (int p = dn.rowptr[i]; p < dn.rowptr[i + 1]; p++) {
        const int k = dn.col[p];
        const double g = dn.G[p], b = dn.B[p];
        ir += g * e[k] - b * f[k];
        ii += g * f[k] + b * e[k];
    }
    if (outage >= 0 && dn.bstatus[outage] && (i == dn.bf[outage] || i == dn.bt[outage])) {
        const double r = dn.br[outage], x = dn.bx[outage], bc = dn.bb[outage], t = dn.btap[outage];
        const double den = r * r + x * x;
        const double ys_re = r / den, ys_im = -x / den;
        const int o = (i == dn.bf[outage]) ? dn.bt[outage] : dn.bf[outage];
        double gs, bs;  // self term of the branch at bus i
        if (i == dn.bf[outage]) {
            gs = ys_re / (t * t);
            bs = (ys_im + 0.5 * bc) / (t * t);
        } else {
            gs = ys_re;
            bs = ys_im + 0.5 * bc;
        }
        const double gm = -ys_re / t, bm = -ys_im / t;  // mutual term
        ir -= gs * e[i] - bs * f[i] + gm * e[o] - bm * f[o];
        ii -= gs * f[i] + bs * e[i] + gm * f[o] + bm * e[o];
    }
    P = e[i] * ir + f[i] * ii;
    Q = f[i] * ir - e[i] * ii;
}

__global__ void k_mismatch_rows(DevNet dn, DevCases dc, const double *vm, const double *ef,
                                double *dp, double *dq, double *maxmis) {
    const int c = blockIdx.y;
    const int nbus = dn.nbus;
    const double *e = ef + (long long)c * 2 * nbus;
    const double *f = e + nbus;
    const int outage = dc.outage[c];
    double mx = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbus; i += gridDim.x * blockDim.x) {
        double P, Q;
        bus_injection(dn, i, outage, e, f, P, Q);
        const int t = dn.btype[i];
        const long long idx = (long long)c * nbus + i;
        const double a = (t != PF_BUS_SLACK) ? dc.Psp[idx] - P : 0.0;
        const double b = (t == PF_BUS_PQ) ? dc.Qsp[idx] - Q : 0.0;
        dp[idx] = a;
        dq[idx] = b;
        double l = fmax(fabs(a), fabs(b));
        if (a != a || b != b) l = __longlong_as_double(0x7ff8000000000000ll);
        mx = (l > mx || l != l) ? l : mx;
    }
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(maxmis + c, mx);
}

// ------------------------------------------------------------ Section III

struct RunArgs {
    DevNet dn;
    DevCases dc;
    DevMat m0, m1;      // B', B''
    const void *F0, *F1;
    const int *fs0, *fs1;
    double tol;
    int max_iter;
    int flat;
    double *vm, *va, *ef, *vec;
    pf_case_result *res;
    int use_smem;
};

// One P or Q half-iteration's mismatch for the block's case: rectangular
// voltages, nodal injections, dP/V (which = 0, B' unknowns) or dQ/V
// (which = 1, B'' unknowns) into the solve vector x in step order.
// Returns the max |mismatch| over all buses (block-uniform).
template <class X>
__device__ double block_mismatch(const RunArgs &a, int c, int which, X *x, double *red) {
    const DevNet &dn = a.dn;
    const int nbus = dn.nbus;
    const double *vm = a.vm + (long long)c * nbus;
    const double *va = a.va + (long long)c * nbus;
    double *e = a.ef + (long long)c * 2 * nbus;
    double *f = e + nbus;
    for (int i = threadIdx.x; i < nbus; i += blockDim.x) {
        double s, co;
        sincos(va[i], &s, &co);
        e[i] = vm[i] * co;
        f[i] = vm[i] * s;
    }
    __syncthreads();
    const int outage = a.dc.outage[c];
    const int *sob = which == 0 ? a.m0.step_of_bus : a.m1.step_of_bus;
    double mx = 0.0;
    for (int i = threadIdx.x; i < nbus; i += blockDim.x) {
        double P, Q;
        bus_injection(dn, i, outage, e, f, P, Q);
        const int t = dn.btype[i];
        const long long idx = (long long)c * nbus + i;
        const double dP = (t != PF_BUS_SLACK) ? a.dc.Psp[idx] - P : 0.0;
        const double dQ = (t == PF_BUS_PQ) ? a.dc.Qsp[idx] - Q : 0.0;
        double l = fmax(fabs(dP), fabs(dQ));
        if (dP != dP || dQ != dQ) l = __longlong_as_double(0x7ff8000000000000ll);
        mx = (l > mx || l != l) ? l : mx;
        const int k = sob[i];
        if (k >= 0) x[k] = X((which == 0 ? dP : dQ) / vm[i]);
    }
    return block_max(mx, red);
}

// The whole fast-decoupled power flow of one case per block (Section III):
// P half-iteration  B' dtheta = dP / V,  Q half-iteration  B'' dV = dQ / V,
// with the mismatch checked before every half-iteration.
template <class T>
__global__ void __launch_bounds__(kRunThreads) k_fdpf(RunArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[33];
    const DevNet &dn = a.dn;
    const int nbus = dn.nbus;
    for (int c = blockIdx.x; c < a.dc.ncase; c += gridDim.x) {
        const int inst = a.dc.inst[c];
        T *x = a.use_smem ? reinterpret_cast<T *>(smem_raw)
                          : reinterpret_cast<T *>(a.vec + (long long)c * 2 * nbus);
        double *vm = a.vm + (long long)c * nbus;
        double *va = a.va + (long long)c * nbus;
        const T *F0 = static_cast<const T *>(a.F0) + (long long)inst * a.m0.stride;
        const T *F1 = static_cast<const T *>(a.F1) + (long long)inst * a.m1.stride;
        int status = PF_ERR_NOT_CONVERGED;
        if (a.fs0[inst] != PF_OK) status = a.fs0[inst];
        else if (a.fs1[inst] != PF_OK) status = a.fs1[inst];
        int iters = 0;
        double mis = INFINITY;
        if (a.flat) {
            for (int i = threadIdx.x; i < nbus; i += blockDim.x) {
                const int t = dn.btype[i];
                vm[i] = (t == PF_BUS_PQ) ? 1.0 : dn.vset[i];
                va[i] = (t == PF_BUS_SLACK) ? dn.va0[i] : 0.0;
            }
            __syncthreads();
        }
        if (status == PF_ERR_NOT_CONVERGED) {
            for (int it = 0; it < a.max_iter; it++) {
                mis = block_mismatch<T>(a, c, 0, x, red);
                if (!isfinite(mis)) { status = PF_ERR_NONFINITE; break; }
                if (mis <= a.tol) { status = PF_OK; break; }
                block_solve<T, T>(a.m0, F0, x);
                for (int k = threadIdx.x; k < a.m0.n; k += blockDim.x)
                    va[a.m0.bus[k]] += double(x[k]);
                __syncthreads();
                iters++;
                mis = block_mismatch<T>(a, c, 1, x, red);
                if (!isfinite(mis)) { status = PF_ERR_NONFINITE; break; }
                if (mis <= a.tol) { status = PF_OK; break; }
                block_solve<T, T>(a.m1, F1, x);
                for (int k = threadIdx.x; k < a.m1.n; k += blockDim.x)
                    vm[a.m1.bus[k]] += double(x[k]);
                __syncthreads();
                iters++;
            }
            if (status == PF_ERR_NOT_CONVERGED) {
                mis = block_mismatch<T>(a, c, 0, x, red);
                if (mis <= a.tol) status = PF_OK;
            }
        }
        if (threadIdx.x == 0) {
            a.res[c].status = status;
            a.res[c].iters = iters;
            a.res[c].ir_steps = 0;
            a.res[c].pad = 0;
            a.res[c].max_mismatch = mis;
        }
        __syncthreads();
    }
}

int grid_for(long long total, int threads) {
    long long b = (total + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return int(b);
}

}  // namespace

// ------------------------------------------------------------ launchers

cudaError_t launch_ybus(const DevNet &dn, cudaStream_t s) {
    k_ybus<<<grid_for(dn.nbus, 128), 128, 0, s>>>(dn);
    return cudaGetLastError();
}

cudaError_t launch_case_spec(const DevNet &dn, const DevCases &dc, const double *ls,
                             cudaStream_t s) {
    k_case_spec<<<grid_for((long long)dc.ncase * dn.nbus, 256), 256, 0, s>>>(dn, dc, ls);
    return cudaGetLastError();
}

cudaError_t launch_assemble_slots(const DevNet &dn, const DevCases &dc, const DevMat &m, int which,
                                  double *A, cudaStream_t s) {
    const long long total = (long long)dc.ninst * (m.n + m.nnz_l);
    k_assemble_slots<<<grid_for(total, 256), 256, 0, s>>>(dn, dc, m, which, A);
    return cudaGetLastError();
}

cudaError_t launch_factor(const DevMat &m, int prec, const double *A, void *F, int ninst,
                          int *fstatus, cudaStream_t s) {
    const int threads = kFactorThreads;
    if (prec == PF_FP64) {
        size_t smem = sizeof(double) * size_t(m.max_col + 1) * (threads / 32);
        cudaFuncSetAttribute(k_factor_ldlt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(smem));
        k_factor_ldlt<double><<<ninst, threads, smem, s>>>(m, A, static_cast<double *>(F), fstatus);
    } else {
        size_t smem = sizeof(float) * size_t(m.max_col + 1) * (threads / 32);
        cudaFuncSetAttribute(k_factor_ldlt<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(smem));
        k_factor_ldlt<float><<<ninst, threads, smem, s>>>(m, A, static_cast<float *>(F), fstatus);
    }
    return cudaGetLastError();
}

cudaError_t launch_solve(const DevMat &m, int prec, const void *F, const int *inst_of_case,
                         double *rhs, int ncase, void *gvec, size_t smem_optin, cudaStream_t s) {
    // The solve vector lives in shared memory when it fits, else in the
    // per-case global scratch gvec ([ncase][2 nbus] doubles).
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    size_t smem = elt * size_t(m.n);
    const int use_smem = smem + 1024 <= smem_optin;
    if (!use_smem) smem = 0;
    if (prec == PF_FP64) {
        cudaFuncSetAttribute(k_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        k_solve<double><<<ncase, kSolveThreads, smem, s>>>(
            m, static_cast<const double *>(F), inst_of_case, rhs, static_cast<double *>(gvec), use_smem);
    } else {
        cudaFuncSetAttribute(k_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        k_solve<float><<<ncase, kSolveThreads, smem, s>>>(
            m, static_cast<const float *>(F), inst_of_case, rhs, static_cast<float *>(gvec), use_smem);
    }
    return cudaGetLastError();
}

cudaError_t launch_mismatch(const DevNet &dn, const DevCases &dc, const double *vm, const double *va,
                            double *dp, double *dq, double *maxmis, double *ef, int ncase,
                            cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(maxmis, 0, sizeof(double) * ncase, s);
    if (e != cudaSuccess) return e;
    k_polar_to_rect<<<grid_for((long long)ncase * dn.nbus, 256), 256, 0, s>>>(dn.nbus, ncase, vm,
                                                                              va, ef);
    dim3 grid((dn.nbus + 255) / 256, ncase);
    k_mismatch_rows<<<grid, 256, 0, s>>>(dn, dc, vm, ef, dp, dq, maxmis);
    return cudaGetLastError();
}

cudaError_t launch_fdpf(const DevNet &dn, const DevCases &dc, const DevMat *m, int prec,
                        const void *F0, const void *F1, const int *fstat0, const int *fstat1,
                        const pf_run_opts &o, double *vm, double *va, double *ef, double *vec,
                        pf_case_result *res, size_t smem_optin, cudaStream_t s) {
    RunArgs a;
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
    a.vm = vm;
    a.va = va;
    a.ef = ef;
    a.vec = vec;
    a.res = res;
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    const int nmax = m[0].n > m[1].n ? m[0].n : m[1].n;
    size_t smem = elt * size_t(nmax);
    a.use_smem = smem <= smem_optin - 1024;
    if (!a.use_smem) smem = 0;
    if (prec == PF_FP64) {
        cudaFuncSetAttribute(k_fdpf<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        k_fdpf<double><<<dc.ncase, kRunThreads, smem, s>>>(a);
    } else {
        cudaFuncSetAttribute(k_fdpf<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        k_fdpf<float><<<dc.ncase, kRunThreads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace gbpf
