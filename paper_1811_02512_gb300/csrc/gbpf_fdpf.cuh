// gbpf_fdpf.cuh -- the power-flow iteration kernels of libgbpf for sm_103a
// (Section III of arxiv 1811.02512): the fast decoupled iteration of one
// case per thread block or per cluster (k_fdpf) and of the grids of a pack
// (k_fdpf_pack), with the nodal mismatch (Section II.A), the staged
// substitutions (Section III.C) with FP64 refinement of FP32 solves, and the
// low-rank form of outage cases.  Included by gbpf_fdpf.cu (launchers, no
// kernel instantiated) and by gbpf_fdpf64.cu / gbpf_fdpf32.cu, which
// instantiate the FP64 and the FP32 kernels in parallel translation units.
#pragma once

#include <cfloat>
#include <cmath>
#include <cstdint>
#include <vector>

#include "gbpf_nr.cuh"

namespace gbpf {

struct RunArgs {
    DevNet dn;
    DevCases dc;
    DevMat m0, m1;  // B', B''
    const void *F0, *F1;
    const void *TV0, *TV1;  // gathered tail values per instance (or null)
    const void *TW0, *TW1;  // tail-inverse values of instance 0 (tail form 3; or null)
    // low-rank outages: outage cases solve with the base factor (instance 0)
    // and the correction x += Z K (x[p0], x[p1]) of their instance (or null)
    const void *Z0, *Z1;     // [ninst][2][n] T
    const double *K0, *K1;   // [ninst][4]
    const double *A0, *A1;  // FP64 assembled values of B', B'' (refinement residuals)
    const int *fs0, *fs1;
    double tol;
    int max_iter;
    int ir_max;
    double ir_tol, ir_abs;
    int flat;
    unsigned spin;
    double *vm, *va;
    double *ef;    // [ncase][4 nbus]: e, f, cos(theta), sin(theta)
    double *iv;    // [ncase][nbus]: 1 / V
    double *xg;    // [ncase][3 nbus]: right-hand side / solution, refined FP64 x, FP32 work
    double *bmax;  // [ncase][16]: per-CTA mismatch maxima, [15] = solve status
    pf_case_result *res;
    int use_smem;
    // FDPF -> NR fallback (Section III): a case that ends unconverged or
    // non-finite restarts from a flat start under Newton-Raphson (nr) in the
    // same launch; its result then reports method PF_NR
    int fallback;
    NrArgs nr;
};


namespace {
// ------------------------------------------------------------ Section III



// One half-iteration's mismatch for case c on the C CTAs of its cluster: each
// CTA owns a slice of buses, forms e + jf from V and the cached cos/sin of
// theta, then (after a cluster barrier) the currents of its rows and writes
// dP/V (which = 0, B' unknowns) or dQ/V (which = 1, B'' unknowns) into the
// exchange vector in level order.  Returns the case maximum (cluster-uniform)
// of |dP| over non-slack and |dQ| over PQ buses when `full`, else of the
// half-iteration's own part only (|dP| or |dQ|): a lower bound of the full
// maximum, so a partial maximum above the tolerance already decides "not
// converged" and only one at or below it needs the full check.  Skipping the
// other part saves FP64 work, which bounds batches on this part.
template <int C>
__device__ double cluster_mismatch(const RunArgs &a, int c, int rank, int which, double *red,
                                   bool full) {
    const DevNet &dn = a.dn;
    const int nbus = dn.nbus;
    const int slice = (nbus + C - 1) / C;
    const int i0 = rank * slice, i1 = min(nbus, i0 + slice);
    const double *vm = a.vm + (long long)c * nbus;
    double *e = a.ef + (long long)c * 4 * nbus;
    double *f = e + nbus;
    const double *cs = e + 2 * nbus;
    const double *sn = e + 3 * nbus;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        e[i] = vm[i] * cs[i];
        f[i] = vm[i] * sn[i];
    }
    cluster_sync<C>();
    const int outage = a.dc.outage[c];
    const int *nob = which == 0 ? a.m0.new_of_bus : a.m1.new_of_bus;
    double *xg = a.xg + (long long)c * 3 * nbus;
    const bool wantP = full || which == 0, wantQ = full || which == 1;
    unsigned long long mx = 0;
    // the next bus index is read a round ahead, off the row's chain
    int inext = i0 + int(threadIdx.x) < i1 ? (C == 1 ? dn.mis_ord[i0 + threadIdx.x] : i0 + int(threadIdx.x)) : 0;
    for (int q = i0 + threadIdx.x; q < i1; q += blockDim.x) {
        const int i = inext;  // a warp's rows of one length
        if (q + int(blockDim.x) < i1) inext = C == 1 ? dn.mis_ord[q + blockDim.x] : q + int(blockDim.x);
        double ir, ii;
        bus_current(dn, i, outage, e, f, ir, ii);
        const int t = dn.btype[i];
        const long long idx = (long long)c * nbus + i;
        double dP = 0.0, dQ = 0.0;
        if (wantP && t != PF_BUS_SLACK) dP = a.dc.Psp[idx] - (e[i] * ir + f[i] * ii);
        if (wantQ && t == PF_BUS_PQ) dQ = a.dc.Qsp[idx] - (f[i] * ir - e[i] * ii);
        const unsigned long long kp = abs_key(dP), kq = abs_key(dQ);
        mx = kp > mx ? kp : mx;
        mx = kq > mx ? kq : mx;
        const int k = nob[i];
        if (k >= 0) xg[k] = (which == 0 ? dP : dQ) * a.iv[(long long)c * nbus + i];
    }
    mx = block_max_key(mx, red);
    if (threadIdx.x == 0) a.bmax[(long long)c * 16 + rank] = __longlong_as_double(static_cast<long long>(mx));
    cluster_sync<C>();
    double m = 0.0;
    for (int r = 0; r < C; r++) m = nan_max(m, a.bmax[(long long)c * 16 + r]);
    return m;
}

// Low-rank outage correction of one case's solve (Woodbury): the outage
// takes the branch's share U S U^T out of the base matrix A (U the unit
// columns of the branch's two buses p0, p1 in level order, absent ones
// skipped), so (A - U S U^T)^-1 b = y + Z K (U^T y) with y = A^-1 b, Z =
// A^-1 U and K = (I - S U^T Z)^-1 S, both computed once per factorisation.
template <class T>
struct LowRank {
    const T *Z = nullptr;     // [2][n] columns A^-1 e_p0, A^-1 e_p1 (null: no correction)
    const double *K = nullptr;  // K00, K01, K10, K11, then S00, S11, S01
    int p0 = -1, p1 = -1;
};

// Row r (p0 or p1) of U S U^T x: the part of the base matrix's row that the
// outaged branch contributes, which the residual b - A x of an outage case
// adds back when it is formed with the base matrix A.
template <class T, class XR>
__device__ __forceinline__ double lowrank_residual(const LowRank<T> &lr, int r, const XR *x) {
    const double s00 = lr.K[4], s11 = lr.K[5], s01 = lr.K[6];
    const double x0 = lr.p0 >= 0 ? double(x[lr.p0]) : 0.0, x1 = lr.p1 >= 0 ? double(x[lr.p1]) : 0.0;
    return r == lr.p0 ? s00 * x0 + s01 * x1 : s01 * x0 + s11 * x1;
}

// Row r of the FP64 residual b - A x (x read as XR and promoted to FP64):
// the diagonal, then the row's off-diagonal entries four at a time (their
// indices and values loaded before the ordered subtractions), then for a
// low-rank outage case the branch's share at its two rows.
template <class T, class XR>
__device__ __forceinline__ double residual_row(const DevMat &m, const double *A, const double *b, const XR *x,
                                               int r, const LowRank<T> &lr) {
    double s = b[r] - A[r] * double(x[r]);
    const int e1 = m.Ap[r + 1];
    int e = m.Ap[r];
    for (; e + 3 < e1; e += 4) {
        const int p0 = m.Apos[e], p1 = m.Apos[e + 1], p2 = m.Apos[e + 2], p3 = m.Apos[e + 3];
        const int j0 = m.Aj[e], j1 = m.Aj[e + 1], j2 = m.Aj[e + 2], j3 = m.Aj[e + 3];
        const double a0 = A[p0], a1 = A[p1], a2 = A[p2], a3 = A[p3];
        const double y0 = double(x[j0]), y1 = double(x[j1]), y2 = double(x[j2]), y3 = double(x[j3]);
        s -= a0 * y0;
        s -= a1 * y1;
        s -= a2 * y2;
        s -= a3 * y3;
    }
    if (e < e1) {
        const int rem = e1 - e;  // 1 to 3 entries
        const int p0 = m.Apos[e], p1 = m.Apos[rem > 1 ? e + 1 : e], p2 = m.Apos[rem > 2 ? e + 2 : e];
        const int j0 = m.Aj[e], j1 = m.Aj[rem > 1 ? e + 1 : e], j2 = m.Aj[rem > 2 ? e + 2 : e];
        const double a0 = A[p0], a1 = A[p1], a2 = A[p2];
        const double y0 = double(x[j0]), y1 = double(x[j1]), y2 = double(x[j2]);
        s -= a0 * y0;
        if (rem > 1) s -= a1 * y1;
        if (rem > 2) s -= a2 * y2;
    }
    if (lr.Z && (r == lr.p0 || r == lr.p1)) s += lowrank_residual(lr, r, x);
    return s;
}

template <class T, class X>
__device__ void lowrank_correct(const LowRank<T> &lr, X *x, int n, double *red) {
    if (!lr.Z) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double y0 = lr.p0 >= 0 ? double(x[lr.p0]) : 0.0, y1 = lr.p1 >= 0 ? double(x[lr.p1]) : 0.0;
        red[0] = lr.K[0] * y0 + lr.K[1] * y1;
        red[1] = lr.K[2] * y0 + lr.K[3] * y1;
    }
    __syncthreads();
    const double s0 = red[0], s1 = red[1];
    for (int r = threadIdx.x; r < n; r += blockDim.x)
        x[r] = X(double(x[r]) + double(lr.Z[r]) * s0 + double(lr.Z[n + r]) * s1);
    __syncthreads();
}

// Solves one matrix of case c in the cluster's CTA 0 (the others wait at the
// following cluster barrier): the exchange vector is staged into shared
// memory, solved with the TMA-staged sweeps and written back.  With an FP32
// factor the solve is refined in FP64: x += solve32(r), r = b - A x with the
// FP64 assembled A, until ||r||inf <= ir_tol ||b||inf or ir_max corrections
// (the refined x lives in the second half of the exchange vector).
template <class T>
__device__ bool rank0_solve(const RunArgs &a, Ring *R, unsigned char *stages, T *xs,
                            const DevMat &m, const T *F, const T *tv, const T *tw, const double *A, int c,
                            double *red, int &ir_steps, const LowRank<T> &lr) {
    const int nbus = a.dn.nbus;
    double *xg = a.xg + (long long)c * 3 * nbus;
    bool ok = true;
    if constexpr (sizeof(T) == sizeof(double)) {
        if (xs) {
            for (int r = threadIdx.x; r < m.n; r += blockDim.x) xs[r] = T(xg[r]);
            __syncthreads();
            ok = block_solve<T, T>(R, stages, m, F, xs, a.spin, tv, tw);
            if (ok) lowrank_correct<T, T>(lr, xs, m.n, red);
            for (int r = threadIdx.x; r < m.n; r += blockDim.x) xg[r] = double(xs[r]);
        } else {
            ok = block_solve<T, double>(R, stages, m, F, xg, a.spin, tv, tw);
            if (ok) lowrank_correct<T, double>(lr, xg, m.n, red);
        }
    } else {
        double *x64 = xg + nbus;
        T *xv = xs ? xs : reinterpret_cast<T *>(x64 + m.n);  // FP32 work vector
        unsigned long long bk = 0;
        for (int r = threadIdx.x; r < m.n; r += blockDim.x) {
            xv[r] = T(xg[r]);
            const unsigned long long k = abs_key(xg[r]);
            bk = k > bk ? k : bk;
        }
        const double bn = __longlong_as_double(static_cast<long long>(block_max_key(bk, red)));
        for (int k = 0;; k++) {
            ok = block_solve<T, T>(R, stages, m, F, xv, a.spin, tv, tw);
            if (!ok) break;
            lowrank_correct<T, T>(lr, xv, m.n, red);
            for (int r = threadIdx.x; r < m.n; r += blockDim.x)
                x64[r] = (k == 0 ? 0.0 : x64[r]) + double(xv[r]);
            __syncthreads();
            if (k >= a.ir_max) break;
            unsigned long long rk = 0;
            for (int r = threadIdx.x; r < m.n; r += blockDim.x) {
                const double s = residual_row<T, double>(m, A, xg, x64, r, lr);
                xv[r] = T(s);
                const unsigned long long q = abs_key(s);
                rk = q > rk ? q : rk;
            }
            const double rn = __longlong_as_double(static_cast<long long>(block_max_key(rk, red)));
            if (!(rn > a.ir_tol * bn) || !(rn > a.ir_abs)) break;
            ir_steps++;
        }
        for (int r = threadIdx.x; r < m.n; r += blockDim.x) xg[r] = x64[r];
    }
    return ok;
}

// The whole fast-decoupled power flow of one case per cluster of C CTAs
// (Section III): P half-iteration B' dtheta = dP / V, Q half-iteration
// B'' dV = dQ / V, with the mismatch checked before every half-iteration.
// With C = 1 every case is one independent block (batches); with C > 1 one
// case spreads its FP64 mismatch over C SMs (single large cases).
template <class T, int C>
__device__ __forceinline__ void fdpf_case(const RunArgs &a, int c, unsigned char *smem_raw,
                                          double *red, Ring &R, bool init_ring) {
    const DevNet &dn = a.dn;
    const int nbus = dn.nbus;
    const int rank = C == 1 ? 0 : int(cluster_rank());
    unsigned char *stages = smem_raw;
    T *xs = a.use_smem ? reinterpret_cast<T *>(smem_raw + kStages * kStageBytes) : nullptr;
    if (init_ring) ring_init(&R);
    const int inst = a.dc.inst[c];
    double *vm = a.vm + (long long)c * nbus;
    double *va = a.va + (long long)c * nbus;
    double *cs = a.ef + (long long)c * 4 * nbus + 2 * nbus;
    double *sn = cs + nbus;
    const double *xg = a.xg + (long long)c * 3 * nbus;
    double *flag = a.bmax + (long long)c * 16 + 15;
    const bool lowrank = a.Z0 != nullptr && inst > 0;
    const int finst = lowrank ? 0 : inst;  // the instance whose factor the solves use
    const T *F0 = static_cast<const T *>(a.F0) + (long long)finst * a.m0.stride;
    const T *F1 = static_cast<const T *>(a.F1) + (long long)finst * a.m1.stride;
    const T *TV0 = a.TV0 ? static_cast<const T *>(a.TV0) + (long long)finst * a.m0.tv_stride : nullptr;
    const T *TV1 = a.TV1 ? static_cast<const T *>(a.TV1) + (long long)finst * a.m1.tv_stride : nullptr;
    const T *TW0 = a.TW0 && finst == 0 ? static_cast<const T *>(a.TW0) : nullptr;
    const T *TW1 = a.TW1 && finst == 0 ? static_cast<const T *>(a.TW1) : nullptr;
    LowRank<T> lr0, lr1;
    if (lowrank) {
        const int e = a.dc.inst_outage[inst];
        lr0.Z = static_cast<const T *>(a.Z0) + (long long)inst * 2 * a.m0.n;
        lr0.K = a.K0 + 8LL * inst;
        lr0.p0 = a.m0.br_slot[3 * e];
        lr0.p1 = a.m0.br_slot[3 * e + 1];
        lr1.Z = static_cast<const T *>(a.Z1) + (long long)inst * 2 * a.m1.n;
        lr1.K = a.K1 + 8LL * inst;
        lr1.p0 = a.m1.br_slot[3 * e];
        lr1.p1 = a.m1.br_slot[3 * e + 1];
    }
    // the FP64 matrices of the refinement residuals: the case's own, or with
    // low-rank outages the base one (the residual adds the branch's share
    // U S U^T back itself: lowrank_residual)
    const double *A0 = a.A0 + (long long)finst * a.m0.stride;
    const double *A1 = a.A1 + (long long)finst * a.m1.stride;
    int ir_steps = 0;
    const int slice = (nbus + C - 1) / C;
    const int i0 = rank * slice, i1 = min(nbus, i0 + slice);
    int status = PF_ERR_NOT_CONVERGED;
    if (a.fs0[finst] != PF_OK) status = a.fs0[finst];
    else if (a.fs1[finst] != PF_OK) status = a.fs1[finst];
    int iters = 0;
    double mis = INFINITY;
    double *iv = a.iv + (long long)c * nbus;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        if (a.flat) {
            const int t = dn.btype[i];
            vm[i] = (t == PF_BUS_PQ) ? 1.0 : dn.vset[i];
            va[i] = (t == PF_BUS_SLACK) ? dn.va0[i] : 0.0;
        }
        sincos(va[i], &sn[i], &cs[i]);
        iv[i] = 1.0 / vm[i];
    }
    cluster_sync<C>();
    // cos/sin of the angles are rotated by each step (small_sincos) rather than
    // re-evaluated, and each half-iteration evaluates only its own part of the
    // mismatch; before a convergence decision the cos/sin are recomputed
    // exactly and the full mismatch re-checked, so the decision is taken on
    // both parts at the exact state
    bool rotated = false;
    auto exact_check = [&](int which) {
        if (rotated)
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) sincos(va[i], &sn[i], &cs[i]);
        rotated = false;
        return cluster_mismatch<C>(a, c, rank, which, red, true);
    };
    if (status == PF_ERR_NOT_CONVERGED) {
        for (int it = 0; it < a.max_iter; it++) {
            mis = cluster_mismatch<C>(a, c, rank, 0, red, false);
            if (mis <= a.tol) mis = exact_check(0);
            if (!isfinite(mis)) { status = PF_ERR_NONFINITE; break; }
            if (mis <= a.tol) { status = PF_OK; break; }
            if (rank == 0) {
                const bool ok = rank0_solve<T>(a, &R, stages, xs, a.m0, F0, TV0, TW0, A0, c, red, ir_steps, lr0);
                if (threadIdx.x == 0) *flag = ok ? 0.0 : 1.0;
            }
            cluster_sync<C>();
            if (*flag != 0.0) { status = PF_ERR_TIMEOUT; break; }
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const int k = a.m0.new_of_bus[i];
                if (k >= 0) {
                    const double d = xg[k];
                    va[i] += d;
                    if (fabs(d) <= kRotMax) {
                        double sd, cd;
                        small_sincos(d, &sd, &cd);
                        const double c0 = cs[i], s0 = sn[i];
                        cs[i] = c0 * cd - s0 * sd;
                        sn[i] = s0 * cd + c0 * sd;
                    } else {
                        sincos(va[i], &sn[i], &cs[i]);
                    }
                }
            }
            rotated = true;
            iters++;
            mis = cluster_mismatch<C>(a, c, rank, 1, red, false);
            if (mis <= a.tol) mis = exact_check(1);
            if (!isfinite(mis)) { status = PF_ERR_NONFINITE; break; }
            if (mis <= a.tol) { status = PF_OK; break; }
            if (rank == 0) {
                const bool ok = rank0_solve<T>(a, &R, stages, xs, a.m1, F1, TV1, TW1, A1, c, red, ir_steps, lr1);
                if (threadIdx.x == 0) *flag = ok ? 0.0 : 1.0;
            }
            cluster_sync<C>();
            if (*flag != 0.0) { status = PF_ERR_TIMEOUT; break; }
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const int k = a.m1.new_of_bus[i];
                if (k >= 0) {
                    vm[i] += xg[k];
                    iv[i] = 1.0 / vm[i];
                }
            }
            iters++;
        }
        if (status == PF_ERR_NOT_CONVERGED) {
            mis = exact_check(0);
            if (mis <= a.tol) status = PF_OK;
        }
    }
    if (a.fallback && (status == PF_ERR_NOT_CONVERGED || status == PF_ERR_NONFINITE)) {
        nr_fallback<T, C>(a.nr, c, rank, smem_raw, red, &R);  // writes the case's result
        return;
    }
    if (rank == 0 && threadIdx.x == 0) {
        a.res[c].status = status;
        a.res[c].iters = iters;
        a.res[c].ir_steps = ir_steps;
        a.res[c].method = PF_FDPF;
        a.res[c].max_mismatch = mis;
    }
    cluster_sync<C>();
}

template <class T, int C>
__global__ void __launch_bounds__(kRunThreads, C == 1 ? 2 : 1) k_fdpf(const __grid_constant__ RunArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[33];
    __shared__ Ring R;
    fdpf_case<T, C>(a, int(blockIdx.x) / C, smem_raw, red, R, true);
}

// Uneven multi-grid batch: one persistent launch over the grids of a pack,
// each grid with its own network, symbolic layout and factors (args[g]).
// Blocks take grids from a counter in the order given by order[] (largest
// first); a grid's solve vector is in shared memory when it fits the
// launch's reservation (args[g].use_smem), else in its global scratch.
template <class T>
__global__ void __launch_bounds__(kRunThreads, 1)
    k_fdpf_pack(const RunArgs *args, const int *order, int ngrid, unsigned *counter) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[33];
    __shared__ Ring R;
    __shared__ int next;
    // the staging ring is initialised once and its phases run on across the
    // grids; after a wait that gave up (ring error) the block runs no more
    // grids and reports those it takes as timed out
    ring_init(&R);
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned q = atomicAdd(counter, 1u);
            next = q < unsigned(ngrid) ? order[q] : -1;
        }
        __syncthreads();
        const int g = next;
        const bool broken = R.err != 0;
        __syncthreads();
        if (g < 0) break;
        if (broken) {
            if (threadIdx.x == 0) {
                args[g].res[0].status = PF_ERR_TIMEOUT;
                args[g].res[0].iters = 0;
                args[g].res[0].ir_steps = 0;
                args[g].res[0].method = PF_FDPF;
                args[g].res[0].max_mismatch = INFINITY;
            }
            continue;
        }
        fdpf_case<T, 1>(args[g], 0, smem_raw, red, R, false);
        __syncthreads();
    }
}

template <class T, int C>
cudaError_t launch_fdpf_t(const RunArgs &a, size_t smem, int threads, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_fdpf<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(a.dc.ncase) * C);
    cfg.blockDim = dim3(unsigned(threads));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    int na = 0;
    if (C > 1) {
        if (C > 8) {
            e = cudaFuncSetAttribute(k_fdpf<T, C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        na = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, k_fdpf<T, C>, a);
}

// Per-precision launchers of the kernels above (gbpf_fdpf64.cu, gbpf_fdpf32.cu).
template <class T>
cudaError_t fdpf_pack_t(const RunArgs *args_dev, const int *order_dev, int ngrid, unsigned *counter_dev,
                        size_t smem, int blocks, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_fdpf_pack<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_fdpf_pack<T><<<blocks, kRunThreads, smem, s>>>(args_dev, order_dev, ngrid, counter_dev);
    return cudaGetLastError();
}

template <class T>
bool fdpf_clusters_fit_t(int C, int ncase, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(C));
    cfg.blockDim = dim3(kRunThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    auto *k = (C == 16) ? k_fdpf<T, 16> : k_fdpf<T, 8>;
    if (C == 16) cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters >= ncase;
}

// threads: of each block (kRunThreads for clusters; 512, 256 or 128 for
// one block per case).
template <class T>
cudaError_t fdpf_run_t(const RunArgs &a, size_t smem, int cluster, int threads, cudaStream_t s) {
    if (cluster >= 16) return launch_fdpf_t<T, 16>(a, smem, kRunThreads, s);
    if (cluster >= 8) return launch_fdpf_t<T, 8>(a, smem, kRunThreads, s);
    return launch_fdpf_t<T, 1>(a, smem, threads, s);
}

}  // namespace

cudaError_t fdpf_pack_f64(const RunArgs *args_dev, const int *order_dev, int ngrid, unsigned *counter_dev,
                          size_t smem, int blocks, cudaStream_t s);
cudaError_t fdpf_pack_f32(const RunArgs *args_dev, const int *order_dev, int ngrid, unsigned *counter_dev,
                          size_t smem, int blocks, cudaStream_t s);
bool fdpf_clusters_fit_f64(int C, int ncase, size_t smem);
bool fdpf_clusters_fit_f32(int C, int ncase, size_t smem);
cudaError_t fdpf_run_f64(const RunArgs &a, size_t smem, int cluster, int threads, cudaStream_t s);
cudaError_t fdpf_run_f32(const RunArgs &a, size_t smem, int cluster, int threads, cudaStream_t s);

}  // namespace gbpf
