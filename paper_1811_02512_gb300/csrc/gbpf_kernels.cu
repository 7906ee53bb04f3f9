// gbpf_kernels.cu -- device kernels of libgbpf for sm_103a (GB300).
//
// Mapping of the paper's two kinds of parallelism (arxiv 1811.02512):
//  * nodal parallelism (Section II.A): one thread per bus row for the
//    admittance matrix (Section III.A, FormMatrixA) and for the P/Q
//    injections and mismatch, spread over the CTAs of a thread-block cluster;
//  * hierarchical parallelism (Section II.B): the levels of the elimination
//    tree run in order, separated by a block barrier; the columns (rows) of
//    one level run in parallel -- one warp per column in the numeric factor
//    (Section III.B), one thread per row/column in the substitutions
//    (Section III.C).
// All factor data is kept in "level order" (elimination steps sorted by
// level), so a level is a contiguous slice of every array.  The substitutions
// stream those slices through a ring of shared-memory stages filled by TMA
// bulk copies (cp.async.bulk + mbarrier), so the dependent chain of a level
// only touches shared memory.
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "gbpf_device.cuh"

#include <vector>

namespace gbpf {

namespace {

// ------------------------------------------------------------ Section III.A

// FormMatrixA (Section III.A), one thread per entry of Y = G + jB: threads
// [0, nbus) the diagonal of bus i -- the pi-model self terms of its
// in-service incident branches (incidence order: ascending branch index)
// plus the bus shunt -- and threads [nbus, nbus + noff) one off-diagonal
// entry each, the negated series admittances of the in-service branches
// between its two buses (ascending branch index).  Every entry is formed in
// registers and written once; a diagonal thread reads the indices of four
// incident branches at a time before their parameters, so a bus of degree
// up to four costs three dependent round trips to memory.  Also writes the
// XB B' (1/x weights) on the same pattern.
__device__ __forceinline__ void ybus_entry(const DevNet &dn, int t) {
    if (t < dn.nbus) {
        const int i = t, q1 = dn.inc_ptr[i + 1];
        double gd = 0.0, bd = 0.0, bpd = 0.0;
        for (int q = dn.inc_ptr[i]; q < q1; q += 4) {
            int e[4], sd[4], on[4];
            double r[4], x[4], b[4], tp[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                e[u] = q + u < q1 ? dn.inc_br[q + u] : -1;
                sd[u] = q + u < q1 ? dn.inc_side[q + u] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                on[u] = 0;
                if (e[u] >= 0) {
                    on[u] = dn.bstatus[e[u]];
                    r[u] = dn.br[e[u]];
                    x[u] = dn.bx[e[u]];
                    b[u] = dn.bb[e[u]];
                    tp[u] = dn.btap[e[u]];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (!on[u]) continue;
                const double den = r[u] * r[u] + x[u] * x[u];
                const double ys_re = r[u] / den, ys_im = -x[u] / den;
                if (sd[u] == 0) {
                    gd += ys_re / (tp[u] * tp[u]);
                    bd += (ys_im + 0.5 * b[u]) / (tp[u] * tp[u]);
                } else {
                    gd += ys_re;
                    bd += ys_im + 0.5 * b[u];
                }
                bpd += 1.0 / x[u];
            }
        }
        const int d = dn.ydiag[i];
        dn.G[d] = gd + dn.gs[i];
        dn.B[d] = bd + dn.bs[i];
        dn.Bp[d] = bpd;
        return;
    }
    const int k = t - dn.nbus;
    if (k >= dn.noff) return;
    const int4 o = dn.yoff[k];
    double g = 0.0, bo = 0.0, bp = 0.0;
    for (int q = o.y; q < o.z; q++) {
        const int e = dn.yoff_br[q];
        if (!dn.bstatus[e]) continue;
        const double r = dn.br[e], x = dn.bx[e], tp = dn.btap[e];
        const double den = r * r + x * x;
        const double ys_re = r / den, ys_im = -x / den;
        g -= ys_re / tp;
        bo -= ys_im / tp;
        bp -= 1.0 / x;
    }
    dn.G[o.x] = g;
    dn.B[o.x] = bo;
    dn.Bp[o.x] = bp;
}

__global__ void k_ybus(DevNet dn) {
    const long long total = (long long)dn.nbus + dn.noff;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x)
        ybus_entry(dn, int(t));
}

// Specified injections of every case: P = pg - pd s, Q = -qd s with the load
// scale s of PQ buses.  Nothing is written when *skip is set (the scales
// failed their check).
__global__ void k_case_spec(DevNet dn, DevCases dc, const double *ls, const int *skip) {
    if (skip && *skip) return;
    const long long total = (long long)dc.ncase * dn.nbus;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = int(idx % dn.nbus);
        const double s = (ls && dn.btype[i] == PF_BUS_PQ) ? ls[idx] : 1.0;
        dc.Psp[idx] = dn.pg[i] - __dmul_rn(dn.pd[i], s);
        dc.Qsp[idx] = -__dmul_rn(dn.qd[i], s);
    }
}

// Contribution of branch e to value slot v (index into the [D | Lc] layout)
// of B' (which = 0) or B'' (which = 1), used to take an outaged branch out.
__device__ double branch_slot_value(const DevNet &dn, const DevMat &m, int which, int e, int v) {
    const int sf = m.br_slot[3 * e], st = m.br_slot[3 * e + 1], sl = m.br_slot[3 * e + 2];
    const double r = dn.br[e], x = dn.bx[e], b = dn.bb[e], t = dn.btap[e];
    if (which == PF_MAT_BP) {
        if (v == sf || v == st) return 1.0 / x;
        if (v == sl) return -1.0 / x;
        return 0.0;
    }
    const double ys_im = -x / (r * r + x * x);
    if (v == sf) return -(ys_im + 0.5 * b) / (t * t);
    if (v == st) return -(ys_im + 0.5 * b);
    if (v == sl) return ys_im / t;
    return 0.0;
}

// Values of B' or B'' of every factor instance in the [D | Lc] layout (fill
// slots zero).
__global__ void k_assemble_slots(DevNet dn, DevCases dc, DevMat m, int which, double *A, int ninst) {
    const int per = m.n + m.nnz;
    const long long total = (long long)ninst * per;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int inst = int(idx / per), s = int(idx % per);
        const int vi = s < m.n ? s : m.offLc + (s - m.n);
        const int src = m.src[s];
        double v = 0.0;
        if (src >= 0) v = (which == PF_MAT_BP) ? dn.Bp[src] : -dn.B[src];
        const int e = dc.inst_outage[inst];
        if (e >= 0 && dn.bstatus[e]) v -= branch_slot_value(dn, m, which, e, vi);
        A[(long long)inst * m.stride + vi] = v;
    }
}

// ------------------------------------------------------------ Section III.B

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until *f == epoch (acquire), polling at most `spin` times with a
// short sleep; gives up early when *abort is raised.  Returns whether the
// flag was seen.
__device__ __forceinline__ bool wait_flag(const unsigned *f, unsigned epoch, unsigned spin,
                                          const unsigned *abort) {
    unsigned it = 0;
    while (ld_acquire_u32(f) != epoch) {
        if (++it > spin || *reinterpret_cast<const volatile unsigned *>(abort)) return false;
        __nanosleep(32);
    }
    return true;
}

// Diagonal maxima of the assembled matrices (the pivot tolerance), status
// reset, and reset of the column counter and abort flag of k_factor_dep.
__global__ void k_factor_prep(DevMat m, const double *A, int *fstatus, FactorSync fs) {
    __shared__ double red[33];
    const int inst = blockIdx.x;
    const double *a = A + (long long)inst * m.stride;
    // four independent loads per thread in flight (the launch waits on this)
    const int st = int(blockDim.x);
    double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
    int j = threadIdx.x;
    for (; j + 3 * st < m.n; j += 4 * st) {
        m0 = fmax(m0, fabs(a[j]));
        m1 = fmax(m1, fabs(a[j + st]));
        m2 = fmax(m2, fabs(a[j + 2 * st]));
        m3 = fmax(m3, fabs(a[j + 3 * st]));
    }
    for (; j < m.n; j += st) m0 = fmax(m0, fabs(a[j]));
    double mx = block_max(fmax(fmax(m0, m1), fmax(m2, m3)), red);
    if (threadIdx.x == 0) {
        fs.amax[inst] = mx;
        fstatus[inst] = PF_OK;
        if (inst == 0) {
            fs.sync[0] = 0u;
            fs.sync[1] = 0u;
        }
    }
}

constexpr int kDepThreads = 256;
constexpr int kDepTargets = 8;   // targets per lane: columns of up to 255 entries
static_assert(32 * kDepTargets == kDepMaxCol + 1, "targets per lane cover the longest column");
constexpr int kDepChunk = 512;   // update terms staged per warp and pass
constexpr int kDepPre = 2;       // targets per lane whose assembled values are read before the waits

// Numeric factor A = L D L^T (Section III.B, left-looking), driven by the
// elimination tree's dependencies instead of level barriers, for every
// instance at once over the whole GPU.  Warps take (column, instance) pairs
// from a global counter in level order; a warp first waits until every
// column k of row c of L is done (its flag holds this factorisation's
// epoch), then evaluates the update terms l_ik d_k l_ck of column c (a
// contiguous range of the gather lists, grouped by target) with the whole
// warp into shared memory, and sums each target's terms with a lane per
// target:
//   d_c = a_cc - sum_k l_ck^2 d_k,   l_ic = (a_ic - sum_k l_ik d_k l_ck) / d_c.
// It writes the column to the column- and row-ordered copies of L and
// publishes its own flag.  Columns are handed out in level order, so every
// column a warp waits for was taken earlier by a running warp: the waits
// always end (each is bounded all the same; a wait that gives up raises the
// abort flag, which ends the others).  The order of operations of every
// entry is fixed, so results are deterministic.  Factor entries of other
// columns are read through L2 (__ldcg): other SMs wrote them in this launch.
// Column c of one instance (a: assembled values, v: factor values, done:
// column flags).  Returns false when a wait gave up (the caller raises the
// abort flag).
template <class T>
__device__ __forceinline__ bool factor_column(const DevMat &m, const double *a, T *v, unsigned *done,
                                              int *fstat, double amax, unsigned epoch, int c,
                                              T *terms, unsigned spin, const unsigned *abort) {
    const int lane = threadIdx.x & 31;
    T *Lc = v + m.offLc;
    // Everything that does not depend on other columns' values is read
    // before the waits, so that after the last dependency is published only
    // the factor values themselves are still to be fetched: the targets'
    // term ranges, the first 128 gather entries and the assembled values of
    // the first 64 targets (columns rarely have more), with their positions
    // in the row-ordered copy.
    const int c0 = m.Cp[c], cnt = m.Cp[c + 1] - c0, tb = c0 + c;
    const int nj = cnt / 32 + 1;  // target slots per lane in use (targets 0..cnt)
    const int gb = m.gp[tb], ge = m.gp[tb + cnt + 1];
    int g_lo[kDepTargets], g_hi[kDepTargets];
    T part[kDepTargets];
    double aval[kDepPre];
    int cpos[kDepPre];
#pragma unroll
    for (int j = 0; j < kDepTargets; j++) {
        const int t = lane + 32 * j;
        g_lo[j] = t <= cnt ? m.gp[tb + t] : 0;
        g_hi[j] = t <= cnt ? m.gp[tb + t + 1] : 0;
        if (j < kDepPre) {
            aval[j] = t <= cnt ? __ldg(t == 0 ? a + c : a + m.offLc + c0 + t - 1) : 0.0;
            cpos[j] = t >= 1 && t <= cnt ? __ldg(m.Cpos + c0 + t - 1) : 0;
        }
        part[j] = T(0);
    }
    int4 e0[4];
#pragma unroll
    for (int u = 0; u < 4; u++)
        if (gb + lane + 32 * u < ge) e0[u] = __ldg(m.gl + gb + lane + 32 * u);
    bool ok = true;
    for (int q = m.Fp[c] + lane; q < m.Fp[c + 1] && ok; q += 32)
        ok = wait_flag(done + m.Fc[q], epoch, spin, abort);
    if (!__all_sync(0xffffffffu, ok)) return false;
    for (int cb = gb; cb < ge; cb += kDepChunk) {
        const int ce = min(ge, cb + kDepChunk);
        // terms of this pass, four per lane in flight
        for (int g0 = cb + lane; g0 < ce; g0 += 128) {
            const bool first = g0 == gb + lane;  // entries read before the waits
            int4 e[4];
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (g0 + 32 * u < ce) e[u] = first ? e0[u] : __ldg(m.gl + g0 + 32 * u);
            T x[4], y[4], z[4];
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (g0 + 32 * u < ce) {
                    x[u] = __ldcg(Lc + e[u].x);
                    y[u] = __ldcg(Lc + e[u].y);
                    z[u] = __ldcg(v + e[u].z);
                }
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (g0 + 32 * u < ce) terms[g0 + 32 * u - cb] = x[u] * (y[u] * z[u]);
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kDepTargets; j++) {
            if (j >= nj) break;  // warp-uniform: no FP64 work for absent targets
            const int lo = max(g_lo[j], cb), hi = min(g_hi[j], ce);
            if constexpr (sizeof(T) == 8) {  // FP64: one chain (no overlap within a warp)
                T s0 = T(0);
                for (int g = lo; g < hi; g++) s0 += terms[g - cb];
                part[j] += s0;
            } else {
                T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
                int g = lo;
                for (; g + 4 <= hi; g += 4) {
                    s0 += terms[g - cb];
                    s1 += terms[g + 1 - cb];
                    s2 += terms[g + 2 - cb];
                    s3 += terms[g + 3 - cb];
                }
                if (g < hi) s0 += terms[g - cb];
                if (g + 1 < hi) s1 += terms[g + 1 - cb];
                if (g + 2 < hi) s2 += terms[g + 2 - cb];
                part[j] += (s0 + s1) + (s2 + s3);
            }
        }
        __syncwarp();
    }
    T val[kDepTargets];
#pragma unroll
    for (int j = 0; j < kDepTargets; j++) {
        if (j >= nj) break;
        const int t = lane + 32 * j;
        const double aj = j < kDepPre ? aval[j] : (t <= cnt ? a[m.offLc + c0 + t - 1] : 0.0);
        val[j] = t <= cnt ? T(aj) - part[j] : T(0);
    }
    const T d = __shfl_sync(0xffffffffu, val[0], 0);
    const T dinv = pivot_recip(d);
    if (lane == 0) {
        v[c] = d;
        v[m.offDi + c] = dinv;
        const double dd = double(d);
        if (!isfinite(dd)) atomicCAS(fstat, PF_OK, PF_ERR_NONFINITE);
        else if (fabs(dd) <= 1e-14 * amax) atomicCAS(fstat, PF_OK, PF_ERR_SINGULAR);
    }
#pragma unroll
    for (int j = 0; j < kDepTargets; j++) {
        if (j >= nj) break;
        const int t = lane + 32 * j;
        if (t >= 1 && t <= cnt) {
            const T l = val[j] * dinv;
            Lc[c0 + t - 1] = l;
            v[m.offLr + (j < kDepPre ? cpos[j] : m.Cpos[c0 + t - 1])] = l;
        }
    }
    // one release by lane 0 after the warp barrier publishes every lane's
    // entries (the barrier orders them before it; a release is cumulative)
    __syncwarp();
    if (lane == 0) st_release_u32(done + c, epoch);
    return true;
}

template <class T>
__global__ void __launch_bounds__(kDepThreads)
    k_factor_dep(DevMat m, const double *A, T *F, int *fstatus, int ninst, FactorSync fs, int ncols) {
    __shared__ T terms_all[kDepThreads / 32][kDepChunk];
    const int lane = threadIdx.x & 31;
    T *terms = terms_all[threadIdx.x >> 5];
    {  // the gather lists and patterns are read once each, in column order:
       // start them (and the assembled values and the column flags) towards
       // the L2 all at once, so that no step of the elimination tree's chain
       // waits for DRAM
        const int part = int(blockIdx.x * blockDim.x + threadIdx.x), parts = int(gridDim.x * blockDim.x);
        l2_prefetch(m.gl, sizeof(int4) * size_t(m.nupd), part, parts);
        l2_prefetch(m.gp, sizeof(int) * size_t(m.n + m.nnz + 1), part, parts);
        l2_prefetch(m.Cp, sizeof(int) * size_t(m.n + 1), part, parts);
        l2_prefetch(m.Fp, sizeof(int) * size_t(m.n + 1), part, parts);
        l2_prefetch(m.Fc, sizeof(int) * size_t(m.nnz), part, parts);
        l2_prefetch(m.Cpos, sizeof(int) * size_t(m.nnz), part, parts);
        l2_prefetch(A, sizeof(double) * size_t(ninst) * size_t(m.stride), part, parts);
        l2_prefetch(fs.done, sizeof(unsigned) * size_t(ninst) * size_t(m.n), part, parts);
    }
    const unsigned total = unsigned(ncols) * unsigned(ninst);
    const unsigned spin = fs.spin ? fs.spin : kDefaultSpin;
    for (;;) {
        unsigned idx = 0;
        if (lane == 0) idx = atomicAdd(fs.sync, 1u);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= total) break;
        const int c = int(idx / unsigned(ninst)), inst = int(idx % unsigned(ninst));
        if (!factor_column<T>(m, A + (long long)inst * m.stride, F + (long long)inst * m.stride,
                              fs.done + (long long)inst * m.n, fstatus + inst, fs.amax[inst], fs.epoch,
                              c, terms, spin, fs.sync + 1) &&
            lane == 0) {
            atomicExch(fs.sync + 1, 1u);
            atomicCAS(fstatus + inst, PF_OK, PF_ERR_TIMEOUT);
        }
    }
}

// The part of every tail target that comes from columns below the tail
// (final once k_factor_dep is done): part = a - sum_{k < t0} L(i,k) D(k)
// L(c,k) over the target's gather terms, one warp per target (lanes stride
// its terms, then a shuffle reduction in lane order), spread over many
// blocks, stored at the target's position in its level (tipos);
// k_factor_tail continues from it.
template <class T>
__global__ void __launch_bounds__(256)
    k_factor_tail_pre(DevMat m, const double *A, const T *F, T *partg) {
    const int inst = blockIdx.y;
    const int k = blockIdx.x * 8 + int(threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (k >= m.ft_ng) return;
    const T *v = F + (long long)inst * m.stride;
    const T *Lc = v + m.offLc;
    const int qe = m.gsplit[k];
    T s = T(0);
    for (int q = m.gp[m.ft_g0 + k] + lane; q < qe; q += 32) {
        const int4 e = m.gl[q];
        s += Lc[e.x] * (Lc[e.y] * v[e.z]);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) partg[(long long)inst * m.ft_ng + m.tipos[k]] = T(A[(long long)inst * m.stride + m.tapos[k]]) - s;
}

// Asynchronous global-to-shared copies of 8 and 16 bytes (both addresses
// aligned to the size), committed as a group and waited for by the issuing
// thread.
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Barrier of the tail factor's level loop: the block's, or the cluster's with
// release / acquire semantics (the values written into other CTAs' shared
// memory before it are visible after it).
template <int C>
__device__ __forceinline__ void tail_barrier() {
    if constexpr (C == 1) __syncthreads();
    else cl_barrier();
}

// The columns [t0, n) of one instance per block (the narrow top of the
// elimination tree), after k_factor_dep has finished the columns below t0
// and k_factor_tail_pre the targets' parts from those columns.
// Shared memory holds the tail's entries, D and 1/D, one partial value per
// gather target, the level table and, double-buffered, the packed terms,
// target descriptors and warp tasks of one level.  Level by level the warps
// take the level's tasks round-robin; a task is 32 / G targets of G lanes
// each (G chosen per target on the host for one term per lane, at most 32),
// so a target with many terms gets many lanes whatever the level's width; each
// target subtracts its terms from tail columns (the level's tables were
// staged while the previous level was computed).  Within the tail the
// entries are kept unnormalised, U(i,c) = L(i,c) D(c), so that an update
// term L(i,k) D(k) L(c,k) is U(i,k) (U(c,k) / D(k)) and a level needs no
// division pass before the next one: one block barrier per level.  L = U / D
// is formed once at the end.  The order of operations of every entry is
// fixed.
//
// With C > 1 one instance runs on a cluster of C CTAs (one per SM, C times
// the FP64 rate of one SM, which bounds a level's terms): every CTA keeps a
// full copy of the tail's values, takes every C-th task of a level, writes
// each value it computes into all C copies over distributed shared memory,
// and a level ends with a cluster barrier instead of the block's.
template <class T, int C>
__global__ void __launch_bounds__(kFactorThreads)
    k_factor_tail(DevMat m, const T *partg, T *F, int *fstatus, const double *amaxv) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int inst = int(blockIdx.x) / C;
    const int rank = C == 1 ? 0 : int(cluster_rank());
    const int bd = int(blockDim.x), tid = int(threadIdx.x);
    const int warp = tid >> 5, lane = tid & 31, nwarps = bd >> 5;
    T *v = F + (long long)inst * m.stride;
    const int tmax = m.ft_tmax, kmax = m.ft_kmax, ntl = m.ntl;
    int4 *lev = reinterpret_cast<int4 *>(smem_raw);  // [2 ntl]
    int4 *tib = lev + 2 * ntl;                        // [2][kmax] target descriptors
    int4 *tkb = tib + 2 * kmax;                       // [2][kmax] warp tasks
    int2 *tbuf = reinterpret_cast<int2 *>(tkb + 2 * kmax);  // [2][tmax]
    T *Ut = reinterpret_cast<T *>(tbuf + 2 * tmax);
    T *Dt = Ut + m.ft_ne;
    T *Di = Dt + m.nt;
    T *part = Di + m.nt;
    // the level loop reads the term, target and task tables once, one level
    // ahead: fetch all of them into the L2 now, so that no level waits for DRAM
    l2_prefetch(m.tterm, sizeof(int2) * size_t(m.ft_tterms), tid, bd);
    l2_prefetch(m.tinfo, sizeof(int4) * size_t(m.ft_ng), tid, bd);
    l2_prefetch(m.ttask, sizeof(int4) * size_t(m.ft_ntask), tid, bd);
    for (int i = tid; i < 2 * ntl; i += bd) lev[i] = m.tlev[i];
    for (int k = tid; k < m.ft_ng; k += bd) part[k] = partg[(long long)inst * m.ft_ng + k];
    {
        const int4 L0 = m.tlev[0], T0 = m.tlev[1];
        for (int i = tid; i < L0.w - L0.z; i += bd) tbuf[i] = m.tterm[L0.z + i];
        for (int i = tid; i < L0.y - L0.x; i += bd) tib[i] = m.tinfo[L0.x + i];
        for (int i = tid; i < T0.w - T0.z; i += bd) tkb[i] = m.ttask[T0.z + i];
    }
    // (a cluster: every CTA has started, so its shared memory may be written)
    tail_barrier<C>();
    int bad = PF_OK;
    const double tol = 1e-14 * amaxv[inst];
    for (int li = 0; li < ntl; li++) {
        const int cur = li & 1;
        const int2 *buf = tbuf + cur * tmax;
        int2 *nbuf = tbuf + (cur ^ 1) * tmax;
        const int4 *ti = tib + cur * kmax;
        int4 *nti = tib + (cur ^ 1) * kmax;
        const int4 *tk = tkb + cur * kmax;
        int4 *ntk = tkb + (cur ^ 1) * kmax;
        const int4 L = lev[2 * li], LT = lev[2 * li + 1];
        const int4 N = li + 1 < ntl ? lev[2 * li + 2] : make_int4(0, 0, 0, 0);
        const int4 NT = li + 1 < ntl ? lev[2 * li + 3] : make_int4(0, 0, 0, 0);
        // the next level's terms, targets and tasks go into the other buffers
        // by asynchronous copies while this level is computed (the barrier
        // that ended the previous level ended every read of those buffers)
        for (int i = tid; i < N.w - N.z; i += bd) cp_async8(nbuf + i, m.tterm + N.z + i);
        for (int i = tid; i < N.y - N.x; i += bd) cp_async16(nti + i, m.tinfo + N.x + i);
        for (int i = tid; i < NT.w - NT.z; i += bd) cp_async16(ntk + i, m.ttask + NT.z + i);
        cp_async_commit();
        // the level's tasks, round-robin over the warps (warp-uniform: the
        // shuffles of a task stay convergent); a warp without a task idles,
        // leaving the FP64 issue slots to the busy ones
        const int ntask = LT.w - LT.z;
        for (int q0 = rank + C * warp; q0 < ntask; q0 += C * nwarps) {
            const int4 task = tk[q0];
            const int G = task.z;
            const int gl = lane & (G - 1), gi = lane / G;
            const bool act = gi < task.y;
            const int j = task.x + gi;
            const int4 info = act ? ti[j] : make_int4(0, 0, 0, 0);
            T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
            int q = info.x + gl;
            const int qe = info.y;
            auto term = [&](int2 u) {
                const unsigned w = unsigned(u.x);
                return Ut[w & 0xffffu] * (Ut[w >> 16] * Di[u.y]);
            };
            T sum;
            if constexpr (sizeof(T) == 8) {
                // FP64: one chain.  A warp's FP64 instructions do not overlap
                // on GB300 (each holds its sub-partition's FP64 unit for about
                // 64 cycles), so split accumulators would only add the
                // instructions that combine them.
                for (; q < qe; q += G) s0 += term(buf[q]);
                sum = s0;
            } else {
                for (; q + 3 * G < qe; q += 4 * G) {
                    s0 += term(buf[q]);
                    s1 += term(buf[q + G]);
                    s2 += term(buf[q + 2 * G]);
                    s3 += term(buf[q + 3 * G]);
                }
                // the last one to three terms of a lane on separate chains too
                if (q < qe) s0 += term(buf[q]);
                if (q + G < qe) s1 += term(buf[q + G]);
                if (q + 2 * G < qe) s2 += term(buf[q + 2 * G]);
                sum = (s0 + s1) + (s2 + s3);
            }
            for (int o = G >> 1; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (!act || gl != 0) continue;
            const T val = part[L.x + j] - sum;
            if (info.z >= 0) {
                Ut[info.z] = val;
                if constexpr (C > 1)
                    for (int r = 1; r < C; r++)
                        st_cl(cl_mapa(smem_u32(Ut + info.z), unsigned((rank + r) % C)), val);
            } else {
                const T dinv = pivot_recip(val);
                Dt[info.w] = val;
                Di[info.w] = dinv;
                if constexpr (C > 1)
                    for (int r = 1; r < C; r++) {
                        const unsigned q = unsigned((rank + r) % C);
                        st_cl(cl_mapa(smem_u32(Dt + info.w), q), val);
                        st_cl(cl_mapa(smem_u32(Di + info.w), q), dinv);
                    }
                const double dd = double(val);
                if (!isfinite(dd)) bad = PF_ERR_NONFINITE;
                else if (fabs(dd) <= tol && bad == PF_OK) bad = PF_ERR_SINGULAR;
            }
        }
        cp_async_wait_all();
        tail_barrier<C>();
    }
    if (bad != PF_OK) atomicCAS(fstatus + inst, PF_OK, bad);
    const int t0 = m.t0, e0 = m.ft_e0;
    for (int c = t0 + rank * bd + tid; c < m.n; c += C * bd) {
        v[c] = Dt[c - t0];
        v[m.offDi + c] = Di[c - t0];
    }
    for (int k = rank * bd + tid; k < m.ft_ng; k += C * bd) {
        const int4 info = m.tinfo[k];
        if (info.z >= 0) {
            const T l = Ut[info.z] / Dt[info.w];
            v[m.offLc + e0 + info.z] = l;
            v[m.offLr + m.Cpos[e0 + info.z]] = l;
        }
    }
}

// Diagonal maxima and status reset of the matrices of a pack (block per job);
// block 0 also resets the pack's column counter and abort flag.
__global__ void k_factor_prep_jobs(const FactorJob *jobs, unsigned *sync) {
    __shared__ double red[33];
    const FactorJob &J = jobs[blockIdx.x];
    double mx = 0.0;
    for (int j = threadIdx.x; j < J.m.n; j += blockDim.x) mx = fmax(mx, fabs(J.A[j]));
    mx = block_max(mx, red);
    if (threadIdx.x == 0) {
        *J.amax = mx;
        *J.fstatus = PF_OK;
        if (blockIdx.x == 0) {
            sync[0] = 0u;
            sync[1] = 0u;
        }
    }
}

// The dependency-driven factor over the matrices of a pack: work items
// (job, column) in an order where every column comes after the columns it
// depends on (levels ascending across all jobs).
template <class T>
__global__ void __launch_bounds__(kDepThreads)
    k_factor_dep_jobs(const FactorJob *jobs, const int2 *items, unsigned nitems, unsigned *sync,
                      unsigned spin) {
    __shared__ T terms_all[kDepThreads / 32][kDepChunk];
    const int lane = threadIdx.x & 31;
    T *terms = terms_all[threadIdx.x >> 5];
    if (!spin) spin = kDefaultSpin;
    for (;;) {
        unsigned idx = 0;
        if (lane == 0) idx = atomicAdd(sync, 1u);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= nitems) break;
        const int2 it = items[idx];
        const FactorJob &J = jobs[it.x];
        if (!factor_column<T>(J.m, J.A, static_cast<T *>(J.F), J.done, J.fstatus, *J.amax, J.epoch, it.y,
                              terms, spin, sync + 1) &&
            lane == 0) {
            atomicExch(sync + 1, 1u);
            atomicCAS(J.fstatus, PF_OK, PF_ERR_TIMEOUT);
        }
    }
}

// Tail values of the matrices of a pack (block-strided per job).
template <class T>
__global__ void k_tail_values_jobs(const FactorJob *jobs) {
    const FactorJob &J = jobs[blockIdx.y];
    if (J.m.npf2 == 0 || !J.TV) return;
    const T *F = static_cast<const T *>(J.F);
    T *TV = static_cast<T *>(J.TV);
    for (int sl = blockIdx.x * blockDim.x + threadIdx.x; sl < J.m.tv_stride; sl += gridDim.x * blockDim.x) {
        const int src = J.m.TVsrc[sl];
        TV[sl] = src >= 0 ? F[src] : T(0);
    }
}

// Block-per-instance form of the same factor (columns of more than 255
// entries): level by level, column c of a level owned by one warp, which
// scatters the updates a_ic -= l_ik d_k l_ck from every descendant column k
// in row c of L (ascending k, so the order of operations is fixed), then
// normalises l_ic = a_ic / d_c.  Columns of one level never write the same
// entry, so no atomics are needed and results are deterministic.  Finally the
// column-ordered L is copied to the row-ordered Lr used by the forward sweep.
template <class T>
__global__ void __launch_bounds__(kFactorThreads)
    k_factor_ldlt(DevMat m, const double *A, T *F, int *fstatus) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[33];
    __shared__ int bad;
    const int inst = blockIdx.x;
    const double *a = A + (long long)inst * m.stride;
    T *v = F + (long long)inst * m.stride;
    T *Lc = v + m.offLc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    T *acc = reinterpret_cast<T *>(smem_raw) + warp * (m.max_col + 1);
    if (threadIdx.x == 0) bad = PF_OK;
    double amax = 0.0;
    for (int j = threadIdx.x; j < m.n; j += blockDim.x) amax = fmax(amax, fabs(a[j]));
    amax = block_max(amax, red);  // its barriers also publish `bad`
    const double piv_tol = 1e-14 * amax;
    const int stride_acc = m.max_col + 1;
    T *fin = reinterpret_cast<T *>(smem_raw) + nwarps * stride_acc;  // narrow levels: reduced column
    for (int lev = 0; lev < m.nlev; lev++) {
        const int cb = m.lvl_ptr[lev], c1 = m.lvl_ptr[lev + 1];
        if (c1 - cb > kNarrowRows) {
            // wide level: one warp per column
            for (int c = cb + warp; c < c1; c += nwarps) {
                const int c0 = m.Cp[c], cnt = m.Cp[c + 1] - c0;
                for (int t = lane; t <= cnt; t += 32)
                    acc[t] = T(t == 0 ? a[c] : a[m.offLc + c0 + t - 1]);
                __syncwarp();
                for (int q = m.Fp[c]; q < m.Fp[c + 1]; q++) {
                    const int k = m.Fc[q], pkc = m.Fpos[q];
                    const T mult = Lc[pkc] * v[k];
                    const int len = m.Cp[k + 1] - pkc, o = m.uoff[q];
                    for (int t = lane; t < len; t += 32) acc[m.umap[o + t]] -= Lc[pkc + t] * mult;
                    __syncwarp();
                }
                const T d = acc[0];
                if (lane == 0) {
                    v[c] = d;
                    v[m.offDi + c] = T(1) / d;
                    const double dd = double(d);
                    if (!isfinite(dd)) atomicCAS(&bad, PF_OK, PF_ERR_NONFINITE);
                    else if (fabs(dd) <= piv_tol) atomicCAS(&bad, PF_OK, PF_ERR_SINGULAR);
                }
                for (int t = lane; t < cnt; t += 32) Lc[c0 + t] = acc[1 + t] / d;
                __syncwarp();
            }
        } else {
            // narrow level: each column with the whole block -- the warps
            // split its update list into per-warp partial sums, reduced in
            // warp order (deterministic)
            for (int c = cb; c < c1; c++) {
                const int c0 = m.Cp[c], cnt = m.Cp[c + 1] - c0;
                for (int t = lane; t <= cnt; t += 32) acc[t] = T(0);
                __syncwarp();
                for (int q = m.Fp[c] + warp; q < m.Fp[c + 1]; q += nwarps) {
                    const int k = m.Fc[q], pkc = m.Fpos[q];
                    const T mult = Lc[pkc] * v[k];
                    const int len = m.Cp[k + 1] - pkc, o = m.uoff[q];
                    for (int t = lane; t < len; t += 32) acc[m.umap[o + t]] += Lc[pkc + t] * mult;
                    __syncwarp();
                }
                __syncthreads();
                for (int t = threadIdx.x; t <= cnt; t += blockDim.x) {
                    T sum = T(t == 0 ? a[c] : a[m.offLc + c0 + t - 1]);
                    const T *part = reinterpret_cast<T *>(smem_raw) + t;
                    for (int w = 0; w < nwarps; w++) sum -= part[w * stride_acc];
                    fin[t] = sum;
                }
                __syncthreads();
                const T d = fin[0];
                if (threadIdx.x == 0) {
                    v[c] = d;
                    v[m.offDi + c] = T(1) / d;
                    const double dd = double(d);
                    if (!isfinite(dd)) atomicCAS(&bad, PF_OK, PF_ERR_NONFINITE);
                    else if (fabs(dd) <= piv_tol) atomicCAS(&bad, PF_OK, PF_ERR_SINGULAR);
                }
                for (int t = threadIdx.x; t < cnt; t += blockDim.x) Lc[c0 + t] = fin[1 + t] / d;
                __syncthreads();
            }
        }
        __syncthreads();
    }
    T *Lr = v + m.offLr;
    for (int q = threadIdx.x; q < m.nnz; q += blockDim.x) Lr[q] = Lc[m.Fpos[q]];
    if (threadIdx.x == 0) fstatus[inst] = bad;
}

// ------------------------------------------------------------ branch flows

// Flows of branch k in case c: S_f = V_f conj(I_f), S_t = V_t conj(I_t) with
// the pi model (series y = 1/(r + jx), charging jb/2 at each end, tap t on
// the from side); zero for the case's outage and out-of-service branches.
__global__ void k_branch_flows(DevNet dn, DevCases dc, const double *vm, const double *va, int ncase,
                               double *flows) {
    const long long total = (long long)ncase * dn.nbr;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int c = int(idx / dn.nbr), k = int(idx - (long long)c * dn.nbr);
        double *o = flows + idx * 4;
        if (!dn.bstatus[k] || dc.outage[c] == k) {
            o[0] = o[1] = o[2] = o[3] = 0.0;
            continue;
        }
        const int f = dn.bf[k], t = dn.bt[k];
        const double *vmc = vm + (long long)c * dn.nbus, *vac = va + (long long)c * dn.nbus;
        double sf, cf, st, ct;
        sincos(vac[f], &sf, &cf);
        sincos(vac[t], &st, &ct);
        const double ef = vmc[f] * cf, ff = vmc[f] * sf, et = vmc[t] * ct, ft = vmc[t] * st;
        const double r = dn.br[k], x = dn.bx[k], den = r * r + x * x;
        const double g = r / den, b = -x / den, bc = 0.5 * dn.bb[k];
        const double tap = dn.btap[k] != 0.0 ? dn.btap[k] : 1.0;
        // I_f = ((g + j(b + bc)) / t^2) V_f - ((g + jb) / t) V_t
        const double gff = g / (tap * tap), bff = (b + bc) / (tap * tap), gft = -g / tap, bft = -b / tap;
        const double ifr = gff * ef - bff * ff + gft * et - bft * ft;
        const double ifi = gff * ff + bff * ef + gft * ft + bft * et;
        // I_t = -((g + jb) / t) V_f + (g + j(b + bc)) V_t
        const double itr = gft * ef - bft * ff + g * et - (b + bc) * ft;
        const double iti = gft * ff + bft * ef + g * ft + (b + bc) * et;
        o[0] = ef * ifr + ff * ifi;
        o[1] = ff * ifr - ef * ifi;
        o[2] = et * itr + ft * iti;
        o[3] = ft * itr - et * iti;
    }
}

// Total active loss of case c (block per case, fixed summation order).
__global__ void k_case_loss(DevNet dn, const double *vm, const double *flows, double *loss) {
    __shared__ double red[32];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int k = threadIdx.x; k < dn.nbr; k += blockDim.x) {
        const double *o = flows + ((long long)c * dn.nbr + k) * 4;
        s += o[0] + o[2];
    }
    const double *vmc = vm + (long long)c * dn.nbus;
    for (int i = threadIdx.x; i < dn.nbus; i += blockDim.x) s += dn.gs[i] * vmc[i] * vmc[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) loss[c] = w;
    }
}

// ------------------------------------------------------------ Section III.C

template <class T>
__global__ void __launch_bounds__(kSolveThreads)
    k_solve(DevMat m, const T *F, const T *TV, const int *inst_of_case, double *rhs, T *gvec,
            int use_smem, int *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Ring R;
    const int c = blockIdx.x;
    const int n = m.n;
    unsigned char *stages = smem_raw;
    T *x = use_smem ? reinterpret_cast<T *>(smem_raw + kStages * kStageBytes)
                    : gvec + (long long)c * 2 * n;
    const T *v = F + (long long)inst_of_case[c] * m.stride;
    double *r = rhs + (long long)c * n;
    ring_init(&R);
    for (int k = threadIdx.x; k < n; k += blockDim.x) x[k] = T(r[m.local[k]]);
    __syncthreads();
    const T *tv = TV ? TV + (long long)inst_of_case[c] * m.tv_stride : nullptr;
    const bool ok = block_solve<T, T>(&R, stages, m, v, x, kDefaultSpin, tv);
    for (int k = threadIdx.x; k < n; k += blockDim.x) r[m.local[k]] = double(x[k]);
    if (threadIdx.x == 0 && !ok) atomicExch(status, PF_ERR_TIMEOUT);
}

// Self-test of the sweeps' give-up path: k_solve's solve of one right-hand
// side with instance 0's factor, with the ring's self-test hooks set (the
// producer issues no piece from stall_at on, or the consumers keep the stage
// of piece hold_at), so that a bounded wait of a sweep runs out.  *status:
// PF_ERR_TIMEOUT when the solve gave up, PF_OK when it completed.
template <class T>
__global__ void __launch_bounds__(kSolveThreads)
    k_selftest_sweep(DevMat m, const T *F, const T *TV, double *rhs, int stall_at, int hold_at,
                     unsigned spin, int *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Ring R;
    T *x = reinterpret_cast<T *>(smem_raw + kStages * kStageBytes);
    ring_init(&R);
    if (threadIdx.x == 0) {
        R.stall_at = stall_at;
        R.hold_at = hold_at;
    }
    for (int k = threadIdx.x; k < m.n; k += blockDim.x) x[k] = T(rhs[m.local[k]]);
    __syncthreads();
    const bool ok = block_solve<T, T>(&R, smem_raw, m, F, x, spin, TV);
    for (int k = threadIdx.x; k < m.n; k += blockDim.x) rhs[m.local[k]] = double(x[k]);
    if (threadIdx.x == 0) *status = ok ? PF_OK : PF_ERR_TIMEOUT;
}

// ------------------------------------------------------------ low-rank outages

// Z = A^-1 U for the outage instances (instance inst >= 1, column col of U =
// the unit vector of the outaged branch's bus p = br_slot[3 e + col], zero
// when that bus is not in the matrix): one block per (instance, column),
// solving with the base factor (instance 0).
template <class T>
__global__ void __launch_bounds__(kSolveThreads)
    k_lowrank_z(DevMat m, DevNet dn, DevCases dc, const T *F, const T *TV, T *Z, T *gvec, int use_smem,
                int *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Ring R;
    const int inst = 1 + int(blockIdx.x) / 2, col = int(blockIdx.x) % 2;
    const int e = dc.inst_outage[inst];
    const int p = (e >= 0 && dn.bstatus[e]) ? m.br_slot[3 * e + col] : -1;
    T *z = Z + ((long long)inst * 2 + col) * m.n;
    if (p < 0) {
        for (int k = threadIdx.x; k < m.n; k += blockDim.x) z[k] = T(0);
        return;
    }
    T *x = use_smem ? reinterpret_cast<T *>(smem_raw + kStages * kStageBytes) : gvec + (long long)blockIdx.x * m.n;
    ring_init(&R);
    for (int k = threadIdx.x; k < m.n; k += blockDim.x) x[k] = T(k == p ? 1 : 0);
    __syncthreads();
    const bool ok = block_solve<T, T>(&R, smem_raw, m, F, x, kDefaultSpin, TV);
    for (int k = threadIdx.x; k < m.n; k += blockDim.x) z[k] = x[k];
    if (threadIdx.x == 0 && !ok) atomicExch(status, PF_ERR_TIMEOUT);
}

// K = (I - S U^T Z)^-1 S of every outage instance (S the branch's share of
// the matrix on its two buses), in FP64, and S itself: Kout[8 inst ..] =
// {K00, K01, K10, K11, S00, S11, S01, 0}; all zero when the branch is already
// out of service.
template <class T>
__global__ void k_lowrank_k(DevMat m, DevNet dn, DevCases dc, int which, const T *Z, double *Kout) {
    for (int inst = 1 + blockIdx.x * blockDim.x + threadIdx.x; inst < dc.ninst; inst += gridDim.x * blockDim.x) {
        double *Kq = Kout + 8LL * inst;
        const int e = dc.inst_outage[inst];
        if (e < 0 || !dn.bstatus[e]) {
            Kq[0] = Kq[1] = Kq[2] = Kq[3] = Kq[4] = Kq[5] = Kq[6] = Kq[7] = 0.0;
            continue;
        }
        const int p0 = m.br_slot[3 * e], p1 = m.br_slot[3 * e + 1], sl = m.br_slot[3 * e + 2];
        const double s00 = p0 >= 0 ? branch_slot_value(dn, m, which, e, p0) : 0.0;
        const double s11 = p1 >= 0 ? branch_slot_value(dn, m, which, e, p1) : 0.0;
        const double s01 = sl >= 0 ? branch_slot_value(dn, m, which, e, sl) : 0.0;
        const T *z0 = Z + (long long)inst * 2 * m.n, *z1 = z0 + m.n;
        // W = U^T Z (W_ij = Z_j at bus p_i)
        const double w00 = p0 >= 0 ? double(z0[p0]) : 0.0, w01 = p0 >= 0 ? double(z1[p0]) : 0.0;
        const double w10 = p1 >= 0 ? double(z0[p1]) : 0.0, w11 = p1 >= 0 ? double(z1[p1]) : 0.0;
        // N = I - S W
        const double n00 = 1.0 - (s00 * w00 + s01 * w10), n01 = -(s00 * w01 + s01 * w11);
        const double n10 = -(s01 * w00 + s11 * w10), n11 = 1.0 - (s01 * w01 + s11 * w11);
        const double det = n00 * n11 - n01 * n10;
        const double i00 = n11 / det, i01 = -n01 / det, i10 = -n10 / det, i11 = n00 / det;
        Kq[0] = i00 * s00 + i01 * s01;
        Kq[1] = i00 * s01 + i01 * s11;
        Kq[2] = i10 * s00 + i11 * s01;
        Kq[3] = i10 * s01 + i11 * s11;
        Kq[4] = s00;  // S itself: the case's matrix is the base one minus U S U^T
        Kq[5] = s11;
        Kq[6] = s01;
        Kq[7] = 0.0;
    }
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
        ef[c * 4 * nbus + i] = vm[idx] * co;
        ef[c * 4 * nbus + nbus + i] = vm[idx] * s;
    }
}

__global__ void k_mismatch_rows(DevNet dn, DevCases dc, const double *ef, double *dp, double *dq,
                                double *maxmis) {
    const int c = blockIdx.y;
    const int nbus = dn.nbus;
    const double *e = ef + (long long)c * 4 * nbus;
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
        mx = nan_max(mx, l);
    }
    mx = warp_max(mx);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(maxmis + c, mx);
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
    k_ybus<<<grid_for((long long)dn.nbus + dn.noff, 128), 128, 0, s>>>(dn);
    return cudaGetLastError();
}

cudaError_t launch_case_spec(const DevNet &dn, const DevCases &dc, const double *ls,
                             cudaStream_t s, const int *skip) {
    k_case_spec<<<grid_for((long long)dc.ncase * dn.nbus, 256), 256, 0, s>>>(dn, dc, ls, skip);
    return cudaGetLastError();
}

// *bad = 1 when any of x[0, n) is not finite (*bad is cleared by the caller).
__global__ void k_finite_check(const double *x, long long n, int *bad) {
    bool ok = true;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        ok &= bool(isfinite(x[i]));
    if (!__all_sync(0xffffffffu, ok) && (threadIdx.x & 31) == 0) *bad = 1;
}

cudaError_t launch_finite_check(const double *x, long long n, int *bad, cudaStream_t s) {
    k_finite_check<<<grid_for(n, 256), 256, 0, s>>>(x, n, bad);
    return cudaGetLastError();
}

cudaError_t launch_lowrank(const DevMat &m, const DevNet &dn, const DevCases &dc, int which, int prec,
                           const void *F, const void *TV, void *Z, double *Kd, void *gvec, int *status,
                           size_t smem_optin, cudaStream_t s) {
    if (dc.ninst < 2) return cudaSuccess;
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    const size_t ring = size_t(kStages) * kStageBytes;
    size_t smem = ring + elt * size_t(m.n);
    const int use_smem = smem + 2048 <= smem_optin;
    if (!use_smem) smem = ring;
    if (m.npf2 == 0) TV = nullptr;
    const int blocks = 2 * (dc.ninst - 1);
    cudaError_t e;
    if (prec == PF_FP64) {
        e = cudaFuncSetAttribute(k_lowrank_z<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        k_lowrank_z<double><<<blocks, kSolveThreads, smem, s>>>(m, dn, dc, static_cast<const double *>(F),
                                                                static_cast<const double *>(TV),
                                                                static_cast<double *>(Z),
                                                                static_cast<double *>(gvec), use_smem, status);
        k_lowrank_k<double><<<(dc.ninst + 127) / 128, 128, 0, s>>>(m, dn, dc, which, static_cast<const double *>(Z), Kd);
    } else {
        e = cudaFuncSetAttribute(k_lowrank_z<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        k_lowrank_z<float><<<blocks, kSolveThreads, smem, s>>>(m, dn, dc, static_cast<const float *>(F),
                                                               static_cast<const float *>(TV),
                                                               static_cast<float *>(Z),
                                                               static_cast<float *>(gvec), use_smem, status);
        k_lowrank_k<float><<<(dc.ninst + 127) / 128, 128, 0, s>>>(m, dn, dc, which, static_cast<const float *>(Z), Kd);
    }
    return cudaGetLastError();
}

cudaError_t launch_branch_flows(const DevNet &dn, const DevCases &dc, const double *vm, const double *va,
                                int ncase, double *flows, double *loss, cudaStream_t s) {
    const long long total = (long long)ncase * dn.nbr;
    k_branch_flows<<<grid_for(total, 256), 256, 0, s>>>(dn, dc, vm, va, ncase, flows);
    k_case_loss<<<ncase, 256, 0, s>>>(dn, vm, flows, loss);
    return cudaGetLastError();
}

cudaError_t launch_assemble_slots(const DevNet &dn, const DevCases &dc, const DevMat &m, int which,
                                  double *A, cudaStream_t s, int ninst) {
    if (ninst < 1 || ninst > dc.ninst) ninst = dc.ninst;
    const long long total = (long long)ninst * (m.n + m.nnz);
    k_assemble_slots<<<grid_for(total, 256), 256, 0, s>>>(dn, dc, m, which, A, ninst);
    return cudaGetLastError();
}

// Values of the scatter-tail schedules and of the tail rows' entries below
// the tail, gathered from the factor of every instance (zero for empty slots).
template <class T>
__global__ void k_tail_values(DevMat m, const T *F, T *TV, int ninst) {
    const long long total = (long long)ninst * m.tv_stride;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long inst = idx / m.tv_stride;
        const int sl = int(idx - inst * m.tv_stride);
        const int src = m.TVsrc[sl];
        TV[idx] = src >= 0 ? F[inst * m.stride + src] : T(0);
    }
}

cudaError_t launch_tail_values(const DevMat &m, int prec, const void *F, void *TV, int ninst,
                               cudaStream_t s) {
    if (m.npf2 == 0 || !TV) return cudaSuccess;
    const long long total = (long long)ninst * m.tv_stride;
    if (prec == PF_FP64)
        k_tail_values<double><<<grid_for(total, 256), 256, 0, s>>>(m, static_cast<const double *>(F),
                                                                   static_cast<double *>(TV), ninst);
    else
        k_tail_values<float><<<grid_for(total, 256), 256, 0, s>>>(m, static_cast<const float *>(F),
                                                                  static_cast<float *>(TV), ninst);
    return cudaGetLastError();
}

cudaError_t launch_factor_jobs(const FactorJob *jobs_dev, int njob, const int2 *items_dev,
                               unsigned nitems, unsigned *sync_dev, int prec, int nsm, cudaStream_t s) {
    k_factor_prep_jobs<<<njob, 256, 0, s>>>(jobs_dev, sync_dev);
    long long blocks = (nitems + kDepThreads / 32 - 1) / (kDepThreads / 32);
    if (blocks > (long long)nsm * 2) blocks = (long long)nsm * 2;
    if (blocks < 1) blocks = 1;
    if (prec == PF_FP64) {
        k_factor_dep_jobs<double><<<int(blocks), kDepThreads, 0, s>>>(jobs_dev, items_dev, nitems, sync_dev, 0u);
        k_tail_values_jobs<double><<<dim3(8, unsigned(njob)), 256, 0, s>>>(jobs_dev);
    } else {
        k_factor_dep_jobs<float><<<int(blocks), kDepThreads, 0, s>>>(jobs_dev, items_dev, nitems, sync_dev, 0u);
        k_tail_values_jobs<float><<<dim3(8, unsigned(njob)), 256, 0, s>>>(jobs_dev);
    }
    return cudaGetLastError();
}

namespace {
// The tail factor of ninst instances: one block each, or (cluster) one
// cluster of kTailCtas CTAs each.
template <class T>
cudaError_t launch_factor_tail(const DevMat &m, const T *partg, T *F, int *fstatus, const double *amax, int ninst,
                               size_t tsmem, bool cluster, cudaStream_t s) {
    if (!cluster) {
        cudaError_t e = cudaFuncSetAttribute(k_factor_tail<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(tsmem));
        if (e != cudaSuccess) return e;
        k_factor_tail<T, 1><<<ninst, kFactorThreads, tsmem, s>>>(m, partg, F, fstatus, amax);
        return cudaGetLastError();
    }
    auto *k = k_factor_tail<T, kTailCtas>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tsmem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(ninst) * kTailCtas);
    cfg.blockDim = dim3(kFactorThreads);
    cfg.dynamicSmemBytes = tsmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kTailCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, m, partg, F, fstatus, amax);
}
}  // namespace

size_t factor_tail_smem(const DevMat &m, int prec) {
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    return elt * (size_t(m.ft_ne) + 2 * size_t(m.nt) + size_t(m.ft_ng)) +
           sizeof(int2) * 2 * size_t(m.ft_tmax > 0 ? m.ft_tmax : 0) +
           sizeof(int4) * 2 * (2 * size_t(m.ft_kmax) + size_t(m.ntl));
}

int factor_tail_clusters(const DevMat &m, int prec) {
    const size_t tsmem = factor_tail_smem(m, prec);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kTailCtas);
    cfg.blockDim = dim3(kFactorThreads);
    cfg.dynamicSmemBytes = tsmem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kTailCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e;
    if (prec == PF_FP64) {
        auto *k = k_factor_tail<double, kTailCtas>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tsmem));
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
    } else {
        auto *k = k_factor_tail<float, kTailCtas>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tsmem));
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_factor(const DevMat &m, int prec, const double *A, void *F, int ninst,
                          int *fstatus, const FactorSync &fs, cudaStream_t s) {
    const long long total = (long long)m.n * ninst;
    const bool dep = fs.mode == 1 || (fs.mode == 0 && ninst < fs.nsm / 2);
    if (dep && m.max_col <= kDepMaxCol && total < (1ll << 31) && fs.done) {
        k_factor_prep<<<ninst, 512, 0, s>>>(m, A, fstatus, fs);
        const size_t tsmem = factor_tail_smem(m, prec);
        const bool tail = fs.tail && m.ft_ng > 0 && m.ft_tmax >= 0 && fs.partg &&
                          tsmem + 1024 <= fs.smem_optin;
        const int ncols = tail ? m.t0 : m.n;
        const int per_sm = fs.blocks_per_sm > 0 && fs.blocks_per_sm < 2 ? fs.blocks_per_sm : 2;  // resident blocks per SM (registers)
        long long blocks = ((long long)ncols * ninst + kDepThreads / 32 - 1) / (kDepThreads / 32);
        if (blocks > (long long)fs.nsm * per_sm) blocks = (long long)fs.nsm * per_sm;
        if (blocks < 1) blocks = 1;
        cudaError_t e = cudaSuccess;
        if (prec == PF_FP64) {
            if (ncols > 0)
                k_factor_dep<double><<<int(blocks), kDepThreads, 0, s>>>(m, A, static_cast<double *>(F),
                                                                          fstatus, ninst, fs, ncols);
            if (tail) {
                k_factor_tail_pre<double><<<dim3(unsigned((m.ft_ng + 7) / 8), unsigned(ninst)), 256, 0, s>>>(
                    m, A, static_cast<const double *>(F), static_cast<double *>(fs.partg));
                e = launch_factor_tail<double>(m, static_cast<const double *>(fs.partg), static_cast<double *>(F),
                                               fstatus, fs.amax, ninst, tsmem, fs.tail_cluster, s);
            }
        } else {
            if (ncols > 0)
                k_factor_dep<float><<<int(blocks), kDepThreads, 0, s>>>(m, A, static_cast<float *>(F),
                                                                         fstatus, ninst, fs, ncols);
            if (tail) {
                k_factor_tail_pre<float><<<dim3(unsigned((m.ft_ng + 7) / 8), unsigned(ninst)), 256, 0, s>>>(
                    m, A, static_cast<const float *>(F), static_cast<float *>(fs.partg));
                e = launch_factor_tail<float>(m, static_cast<const float *>(fs.partg), static_cast<float *>(F),
                                              fstatus, fs.amax, ninst, tsmem, fs.tail_cluster, s);
            }
        }
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    const int threads = kFactorThreads;
    if (prec == PF_FP64) {
        size_t smem = sizeof(double) * size_t(m.max_col + 1) * (threads / 32 + 1);
        cudaFuncSetAttribute(k_factor_ldlt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(smem));
        k_factor_ldlt<double><<<ninst, threads, smem, s>>>(m, A, static_cast<double *>(F), fstatus);
    } else {
        size_t smem = sizeof(float) * size_t(m.max_col + 1) * (threads / 32 + 1);
        cudaFuncSetAttribute(k_factor_ldlt<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(smem));
        k_factor_ldlt<float><<<ninst, threads, smem, s>>>(m, A, static_cast<float *>(F), fstatus);
    }
    return cudaGetLastError();
}

cudaError_t launch_solve(const DevMat &m, int prec, const void *F, const void *TV,
                         const int *inst_of_case, double *rhs, int ncase, void *gvec, int *status,
                         size_t smem_optin, cudaStream_t s) {
    if (m.npf2 == 0) TV = nullptr;
    // The solve vector lives in shared memory after the staging ring when it
    // fits, else in the per-case global scratch gvec ([ncase][2 nbus] doubles).
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    const size_t ring = size_t(kStages) * kStageBytes;
    size_t smem = ring + elt * size_t(m.n);
    const int use_smem = smem + 2048 <= smem_optin;
    if (!use_smem) smem = ring;
    if (prec == PF_FP64) {
        cudaFuncSetAttribute(k_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        k_solve<double><<<ncase, kSolveThreads, smem, s>>>(m, static_cast<const double *>(F),
                                                            static_cast<const double *>(TV),
                                                            inst_of_case, rhs,
                                                            static_cast<double *>(gvec), use_smem,
                                                            status);
    } else {
        cudaFuncSetAttribute(k_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        k_solve<float><<<ncase, kSolveThreads, smem, s>>>(m, static_cast<const float *>(F),
                                                          static_cast<const float *>(TV),
                                                          inst_of_case, rhs,
                                                          static_cast<float *>(gvec), use_smem,
                                                          status);
    }
    return cudaGetLastError();
}

cudaError_t launch_selftest_sweep(const DevMat &m, int prec, const void *F, const void *TV, double *rhs,
                                  int stall_at, int hold_at, unsigned spin, int *status,
                                  size_t smem_optin, cudaStream_t s) {
    if (m.npf2 == 0) TV = nullptr;
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    const size_t smem = size_t(kStages) * kStageBytes + elt * size_t(m.n);
    if (smem + 2048 > smem_optin) return cudaErrorInvalidValue;
    cudaError_t e;
    if (prec == PF_FP64) {
        e = cudaFuncSetAttribute(k_selftest_sweep<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        k_selftest_sweep<double><<<1, kSolveThreads, smem, s>>>(m, static_cast<const double *>(F),
                                                                static_cast<const double *>(TV), rhs,
                                                                stall_at, hold_at, spin, status);
    } else {
        e = cudaFuncSetAttribute(k_selftest_sweep<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        k_selftest_sweep<float><<<1, kSolveThreads, smem, s>>>(m, static_cast<const float *>(F),
                                                               static_cast<const float *>(TV), rhs,
                                                               stall_at, hold_at, spin, status);
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
    k_mismatch_rows<<<grid, 256, 0, s>>>(dn, dc, ef, dp, dq, maxmis);
    return cudaGetLastError();
}

}  // namespace gbpf

// Self-test hook of small_sincos: s[i], c[i] for x[i] (|x| <= 0.2), so tests
// can compare it with the CUDA math library's sincos on the device.
namespace {
__global__ void k_small_sincos(const double *x, double *s, double *c, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) gbpf::small_sincos(x[i], s + i, c + i);
}
__global__ void k_ref_sincos(const double *x, double *s, double *c, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) sincos(x[i], s + i, c + i);
}
}  // namespace

// Self-test hook of the bounded waits: an mbarrier on which nothing arrives
// and a done flag that nothing sets must both give up after their limit and
// report it (out[0], out[1] = 1 when the wait gave up), with the cycles spent
// (out[2], out[3]).
namespace {
__global__ void k_selftest_waits(long long *out, unsigned limit, unsigned *flag, unsigned *abort) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        gbpf::mbar_init(&bar, 1);
        gbpf::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t0 = clock64();
        const bool got = gbpf::mbar_wait_bounded(&bar, 0u, limit);
        out[0] = got ? 0 : 1;
        out[2] = clock64() - t0;
        t0 = clock64();
        const bool seen = gbpf::wait_flag(flag, 1u, limit, abort);
        out[1] = seen ? 0 : 1;
        out[3] = clock64() - t0;
    }
}
}  // namespace

extern "C" int gbpf_selftest_waits(unsigned limit, long long *out_host) {
    long long *out = nullptr;
    unsigned *flags = nullptr;
    if (cudaMalloc(&out, 4 * sizeof(long long)) != cudaSuccess) return 1;
    if (cudaMalloc(&flags, 2 * sizeof(unsigned)) != cudaSuccess) {
        cudaFree(out);
        return 1;
    }
    cudaMemset(flags, 0, 2 * sizeof(unsigned));
    k_selftest_waits<<<1, 32>>>(out, limit, flags, flags + 1);
    cudaError_t e = cudaMemcpy(out_host, out, 4 * sizeof(long long), cudaMemcpyDeviceToHost);
    cudaFree(out);
    cudaFree(flags);
    return e == cudaSuccess ? 0 : 1;
}

namespace gbpf {
namespace {
__global__ void k_pivot_recip(const double *v, double *r, double *ref, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        r[i] = pivot_recip(v[i]);
        ref[i] = 1.0 / v[i];
    }
}
}  // namespace
}  // namespace gbpf

// Test hook (needs a GPU): the pivots' reciprocal (Newton from the FP32
// reciprocal) and CUDA's FP64 division 1 / v of n device values.  Returns 0,
// 1 for a bad argument or a failed launch.
extern "C" int gbpf_selftest_pivot_recip(const double *v_dev, double *r_dev, double *ref_dev, int n) {
    if (n < 1) return 1;
    gbpf::k_pivot_recip<<<(n + 255) / 256, 256>>>(v_dev, r_dev, ref_dev, n);
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}

extern "C" int gbpf_selftest_small_sincos(const double *x_dev, double *s_dev, double *c_dev,
                                          double *s_ref_dev, double *c_ref_dev, int n) {
    if (n < 1) return 1;
    k_small_sincos<<<(n + 255) / 256, 256>>>(x_dev, s_dev, c_dev, n);
    k_ref_sincos<<<(n + 255) / 256, 256>>>(x_dev, s_ref_dev, c_ref_dev, n);
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}
