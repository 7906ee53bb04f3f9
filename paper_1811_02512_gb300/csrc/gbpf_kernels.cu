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

#include "gbpf_internal.h"

namespace gbpf {

namespace {

constexpr int kFactorThreads = 512;
constexpr int kSolveThreads = 512;
constexpr int kRunThreads = 512;
constexpr int kStages = 4;                  // ring depth of the staged sweeps
constexpr int kStageBytes = kPieceBytes;    // one piece per stage
constexpr unsigned kDefaultSpin = 1u << 22; // bound of every mbarrier wait

// ------------------------------------------------------------ small helpers

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

__device__ __forceinline__ double nan_max(double a, double b) { return (b > a || b != b) ? b : a; }

// Atomic maximum of a non-negative double through its bit pattern (IEEE order
// of non-negative doubles equals integer order; NaN patterns sort above Inf).
__device__ void atomic_max_nonneg(double *addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long *>(addr),
              static_cast<unsigned long long>(__double_as_longlong(v)));
}

// ------------------------------------------------------------ TMA / mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bulk copy global -> this CTA's shared memory, completion counted on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of `bar`, giving up after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned limit) {
    for (unsigned i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ------------------------------------------------------------ cluster barrier

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

template <int C>
__device__ __forceinline__ void cluster_sync() {
    if constexpr (C == 1) {
        __syncthreads();
    } else {
        __threadfence();
        asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::
                         : "memory");
    }
}

// ------------------------------------------------------------ staged sweeps

// Shared-memory ring of kStages stages; each stage holds one piece: row
// pointers, indices and values of a run of rows of one level.
struct Ring {
    uint64_t bar[kStages];
    int hdr[kStages][16]; // r0, r1, e0, p_lo, i_lo, v_lo, idx off, val off, mode, run_end,
                          // diag off (-1: none), d_lo, level-pointer off, lp_lo, l0, l1
    int err;              // set when a wait gave up
    unsigned gcount;      // pieces consumed so far (phase bookkeeping)
};

__device__ void ring_init(Ring *R) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) mbar_init(&R->bar[s], 1);
        R->err = 0;
        R->gcount = 0;
        fence_mbar_init();
    }
    __syncthreads();
}

// Issues piece `pc` of a sweep over (ptr, idx, val) into stage `st`.
// Called by one thread.  Ranges are widened to 16-byte boundaries; the arrays
// are padded so the widened ranges stay inside their allocations.
template <class T>
__device__ void ring_issue(Ring *R, unsigned char *stages, int st, const Piece &pc, const int *ptr,
                           const int *idx, const T *val, const T *dinv, const int *lvl_ptr) {
    constexpr int V = 16 / int(sizeof(T));
    const int p_lo = pc.r0 & ~3, p_hi = (pc.r1 + 1 + 3) & ~3;
    const int i_lo = pc.e0 & ~3, i_hi = (pc.e1 + 3) & ~3;
    const int v_lo = pc.e0 & ~(V - 1), v_hi = (pc.e1 + V - 1) & ~(V - 1);
    const int d_lo = pc.r0 & ~(V - 1), d_hi = (pc.r1 + V - 1) & ~(V - 1);
    const uint32_t pbytes = uint32_t(p_hi - p_lo) * 4u;
    const uint32_t ibytes = pc.e1 > pc.e0 ? uint32_t(i_hi - i_lo) * 4u : 0u;
    const uint32_t vbytes = pc.e1 > pc.e0 ? uint32_t(v_hi - v_lo) * uint32_t(sizeof(T)) : 0u;
    const uint32_t dbytes = dinv ? uint32_t(d_hi - d_lo) * uint32_t(sizeof(T)) : 0u;
    const int lp_lo = pc.l0 & ~3, lp_hi = (pc.l1 + 2 + 3) & ~3;
    const uint32_t lbytes = pc.mode == 2 ? uint32_t(lp_hi - lp_lo) * 4u : 0u;
    const int ioff = int(pbytes);
    const int voff = ioff + int(ibytes);
    const int doff = voff + int(vbytes);
    const int loff = doff + int(dbytes);
    int *h = R->hdr[st];
    h[0] = pc.r0; h[1] = pc.r1; h[2] = pc.e0; h[3] = p_lo; h[4] = i_lo; h[5] = v_lo;
    h[6] = ioff; h[7] = voff; h[8] = pc.mode; h[9] = pc.run_end;
    h[10] = dinv ? doff : -1; h[11] = d_lo; h[12] = loff; h[13] = lp_lo; h[14] = pc.l0; h[15] = pc.l1;
    unsigned char *dst = stages + size_t(st) * kStageBytes;
    fence_proxy_async();
    mbar_arrive_expect_tx(&R->bar[st], pbytes + ibytes + vbytes + dbytes + lbytes);
    tma_g2s(dst, ptr + p_lo, pbytes, &R->bar[st]);
    if (ibytes) {
        tma_g2s(dst + ioff, idx + i_lo, ibytes, &R->bar[st]);
        tma_g2s(dst + voff, val + v_lo, vbytes, &R->bar[st]);
    }
    if (dbytes) tma_g2s(dst + doff, dinv + d_lo, dbytes, &R->bar[st]);
    if (lbytes) tma_g2s(dst + loff, lvl_ptr + lp_lo, lbytes, &R->bar[st]);
}

template <class X>
__device__ __forceinline__ X warp_sum(X v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Rows of one staged piece: x[r] = x[r] (* dinv[r] when the piece carries
// the inverse diagonal, i.e. back substitution with the normalisation of
// Eq. 4 fused in) - sum_e val[e] x[idx[e]].  mode 0: thread per row; mode 1:
// warp per row over all warps; mode 2: the calling warp alone, split into
// groups of 32/R lanes for the R <= 16 rows of the piece.  Entries of a row
// are spread over the lanes of its warp or group and summed by shuffles.
template <class T, class X>
__device__ __forceinline__ void piece_rows(const int *h, const unsigned char *base, X *x, int mode,
                                           int first, int stride) {
    const int *P = reinterpret_cast<const int *>(base);
    const int *I = reinterpret_cast<const int *>(base + h[6]);
    const T *Vv = reinterpret_cast<const T *>(base + h[7]);
    const T *Dv = h[10] >= 0 ? reinterpret_cast<const T *>(base + h[10]) : nullptr;
    const int r0 = h[0], rows = h[1] - h[0], p_lo = h[3], i_lo = h[4], v_lo = h[5], d_lo = h[11];
    if (mode == 0) {
        for (int i = first; i < rows; i += stride) {
            const int r = r0 + i;
            const int a = P[r - p_lo], b = P[r + 1 - p_lo];
            X s = Dv ? x[r] * X(Dv[r - d_lo]) : x[r];
            for (int e = a; e < b; e++) s -= X(Vv[e - v_lo]) * x[I[e - i_lo]];
            x[r] = s;
        }
    } else if (mode == 1) {
        const int lane = threadIdx.x & 31;
        for (int i = first; i < rows; i += stride) {
            const int r = r0 + i;
            const int a = P[r - p_lo], b = P[r + 1 - p_lo];
            X s = X(0);
            for (int e = a + lane; e < b; e += 32) s += X(Vv[e - v_lo]) * x[I[e - i_lo]];
            s = warp_sum(s);
            if (lane == 0) x[r] = (Dv ? x[r] * X(Dv[r - d_lo]) : x[r]) - s;
        }
    } else {
        // whole narrow levels l0..l1: ascending in the forward sweep,
        // descending in the backward sweep (the one carrying the diagonal)
        const int lane = threadIdx.x & 31;
        const int *LP = reinterpret_cast<const int *>(base + h[12]) - h[13];
        const int l0 = h[14], l1 = h[15];
        const bool down = Dv != nullptr;
        for (int li = 0; li <= l1 - l0; li++) {
            const int l = down ? l1 - li : l0 + li;
            const int lr0 = LP[l], lrows = LP[l + 1] - LP[l];
            const int gsz = lrows <= 1 ? 32 : lrows <= 2 ? 16 : lrows <= 4 ? 8 : lrows <= 8 ? 4 : 2;
            const int grp = lane / gsz, gl = lane % gsz;
            for (int i0 = 0; i0 < lrows; i0 += 32 / gsz) {
                const int i = i0 + grp;
                X s = X(0);
                int r = -1;
                if (i < lrows) {
                    r = lr0 + i;
                    const int a = P[r - p_lo], b = P[r + 1 - p_lo];
                    for (int e = a + gl; e < b; e += gsz) s += X(Vv[e - v_lo]) * x[I[e - i_lo]];
                }
                for (int o = gsz >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (r >= 0 && gl == 0) x[r] = (Dv ? x[r] * X(Dv[r - d_lo]) : x[r]) - s;
            }
            __syncwarp();
        }
    }
    (void)r0;
    (void)rows;
}

// One substitution sweep: for every piece in order, every row r of the piece
// gets x[r] -= sum_e val[e] * x[idx[e]] over its entries.  Pieces of the same
// level are independent.  Block-wide pieces end with a block barrier that
// also releases their stage; runs of narrow levels (mode 2) are consumed by
// warp 0 alone with warp barriers while the other warps wait at the end of
// the run.  Returns false if a wait gave up (then no copy is left in flight).
template <class T, class X>
__device__ bool staged_sweep(Ring *R, unsigned char *stages, const Piece *pieces, int np,
                             const int *ptr, const int *idx, const T *val, const T *dinv,
                             const int *lvl_ptr, X *x, unsigned spin) {
    const unsigned g0 = R->gcount;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    Piece next{};     // thread 0: descriptor of the next piece to issue, loaded ahead
    int issued = 0;   // thread 0: pieces issued so far in this sweep
    if (threadIdx.x == 0) {
        const int pre = np < kStages ? np : kStages;
        for (int j = 0; j < pre; j++)
            ring_issue<T>(R, stages, int((g0 + j) % kStages), pieces[j], ptr, idx, val, dinv, lvl_ptr);
        issued = pre;
        if (kStages < np) next = pieces[kStages];
    }
    auto issue_after = [&](int j) {  // stage of piece j is free: refill it with j + kStages
        if (j + kStages < np) {
            ring_issue<T>(R, stages, int((g0 + j) % kStages), next, ptr, idx, val, dinv, lvl_ptr);
            issued = j + kStages + 1;
            if (j + kStages + 1 < np) next = pieces[j + kStages + 1];
        }
    };
    bool ok = true;
    int j = 0;
    while (j < np) {
        const unsigned g = g0 + unsigned(j);
        const int st = int(g % kStages);
        if (!mbar_wait_bounded(&R->bar[st], (g / kStages) & 1u, spin)) atomicExch(&R->err, 1);
        const int *h = R->hdr[st];
        const int mode = h[8];
        if (mode == 2) {
            const int jr = h[9];
            __syncthreads();  // every warp has read this header before warp 0 refills the stage
            if (warp == 0) {
                for (int jj = j; jj < jr; jj++) {
                    const unsigned gg = g0 + unsigned(jj);
                    const int s2 = int(gg % kStages);
                    if (jj > j && !mbar_wait_bounded(&R->bar[s2], (gg / kStages) & 1u, spin))
                        atomicExch(&R->err, 1);
                    __syncwarp();
                    if (R->err) break;
                    piece_rows<T, X>(R->hdr[s2], stages + size_t(s2) * kStageBytes, x, 2, 0, 1);
                    __syncwarp();
                    if (lane == 0) issue_after(jj);
                }
            }
            __syncthreads();
            if (R->err) { ok = false; break; }
            j = jr;
        } else {
            if (!R->err)
                piece_rows<T, X>(h, stages + size_t(st) * kStageBytes, x, mode,
                                 mode == 0 ? int(threadIdx.x) : warp,
                                 mode == 0 ? int(blockDim.x) : nwarps);
            __syncthreads();
            if (R->err) { ok = false; break; }
            if (threadIdx.x == 0) issue_after(j);
            j++;
        }
    }
    if (!ok && threadIdx.x == 0) {
        // drain: at most the last kStages issued pieces can still be in flight
        for (int q = (issued > kStages ? issued - kStages : 0); q < issued; q++) {
            const unsigned gq = g0 + unsigned(q);
            mbar_wait_bounded(&R->bar[gq % kStages], (gq / kStages) & 1u, spin);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) R->gcount = g0 + unsigned(np);
    __syncthreads();
    return ok;
}

// L D L^T x = x in place (level order): forward substitution over the rows
// of L (levels ascending), then back substitution over the columns of L
// (levels descending) with the normalisation y = z / d of Eq. 4 fused in as
// a multiplication by the stored inverse diagonal.
template <class T, class X>
__device__ bool block_solve(Ring *R, unsigned char *stages, const DevMat &m, const T *F, X *x,
                            unsigned spin) {
    if (!staged_sweep<T, X>(R, stages, m.pf, m.npf, m.Fp, m.Fc, F + m.offLr, nullptr, m.lvl_ptr, x,
                            spin))
        return false;
    return staged_sweep<T, X>(R, stages, m.pb, m.npb, m.Cp, m.Cr, F + m.offLc, F + m.offDi,
                              m.lvl_ptr, x, spin);
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
__global__ void k_assemble_slots(DevNet dn, DevCases dc, DevMat m, int which, double *A) {
    const int per = m.n + m.nnz;
    const long long total = (long long)dc.ninst * per;
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

// Numeric factor A = L D L^T of one instance per block, left-looking, level by
// level (FactorizeGraphA).  Column c of a level is owned by one warp: it
// gathers the updates a_ic -= l_ik d_k l_ck from every descendant column k in
// row c of L (ascending k, so the order of operations is fixed), then
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

// ------------------------------------------------------------ Section III.C

template <class T>
__global__ void __launch_bounds__(kSolveThreads)
    k_solve(DevMat m, const T *F, const int *inst_of_case, double *rhs, T *gvec, int use_smem,
            int *status) {
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
    const bool ok = block_solve<T, T>(&R, stages, m, v, x, kDefaultSpin);
    for (int k = threadIdx.x; k < n; k += blockDim.x) r[m.local[k]] = double(x[k]);
    if (threadIdx.x == 0 && !ok) atomicExch(status, PF_ERR_TIMEOUT);
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

// ------------------------------------------------------------ Section III

struct RunArgs {
    DevNet dn;
    DevCases dc;
    DevMat m0, m1;  // B', B''
    const void *F0, *F1;
    const int *fs0, *fs1;
    double tol;
    int max_iter;
    int flat;
    unsigned spin;
    double *vm, *va;
    double *ef;    // [ncase][4 nbus]: e, f, cos(theta), sin(theta)
    double *xg;    // [ncase][2 nbus]: right-hand side / solution exchange
    double *bmax;  // [ncase][16]: per-CTA mismatch maxima, [15] = solve status
    pf_case_result *res;
    int use_smem;
};

// One half-iteration's mismatch for case c on the C CTAs of its cluster: each
// CTA owns a slice of buses, forms e + jf from V and the cached cos/sin of
// theta, then (after a cluster barrier) the injections of its rows and writes
// dP/V (which = 0, B' unknowns) or dQ/V (which = 1, B'' unknowns) into the
// exchange vector in level order.  Returns the case maximum (cluster-uniform).
template <int C>
__device__ double cluster_mismatch(const RunArgs &a, int c, int rank, int which, double *red) {
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
    double *xg = a.xg + (long long)c * 2 * nbus;
    double mx = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        double P, Q;
        bus_injection(dn, i, outage, e, f, P, Q);
        const int t = dn.btype[i];
        const long long idx = (long long)c * nbus + i;
        const double dP = (t != PF_BUS_SLACK) ? a.dc.Psp[idx] - P : 0.0;
        const double dQ = (t == PF_BUS_PQ) ? a.dc.Qsp[idx] - Q : 0.0;
        double l = fmax(fabs(dP), fabs(dQ));
        if (dP != dP || dQ != dQ) l = __longlong_as_double(0x7ff8000000000000ll);
        mx = nan_max(mx, l);
        const int k = nob[i];
        if (k >= 0) xg[k] = (which == 0 ? dP : dQ) / vm[i];
    }
    mx = block_max(mx, red);
    if (threadIdx.x == 0) a.bmax[(long long)c * 16 + rank] = mx;
    cluster_sync<C>();
    double m = 0.0;
    for (int r = 0; r < C; r++) m = nan_max(m, a.bmax[(long long)c * 16 + r]);
    return m;
}

// Solves one matrix of case c in the cluster's CTA 0 (the others wait at the
// following cluster barrier): the exchange vector is staged into shared
// memory, solved with the TMA-staged sweeps and written back.
template <class T>
__device__ bool rank0_solve(const RunArgs &a, Ring *R, unsigned char *stages, T *xs,
                            const DevMat &m, const T *F, int c) {
    double *xg = a.xg + (long long)c * 2 * a.dn.nbus;
    bool ok;
    if (xs) {
        for (int r = threadIdx.x; r < m.n; r += blockDim.x) xs[r] = T(xg[r]);
        __syncthreads();
        ok = block_solve<T, T>(R, stages, m, F, xs, a.spin);
        for (int r = threadIdx.x; r < m.n; r += blockDim.x) xg[r] = double(xs[r]);
    } else {
        ok = block_solve<T, double>(R, stages, m, F, xg, a.spin);
    }
    return ok;
}

// The whole fast-decoupled power flow of one case per cluster of C CTAs
// (Section III): P half-iteration B' dtheta = dP / V, Q half-iteration
// B'' dV = dQ / V, with the mismatch checked before every half-iteration.
// With C = 1 every case is one independent block (batches); with C > 1 one
// case spreads its FP64 mismatch over C SMs (single large cases).
template <class T, int C>
__global__ void __launch_bounds__(kRunThreads) k_fdpf(RunArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[33];
    __shared__ Ring R;
    const DevNet &dn = a.dn;
    const int nbus = dn.nbus;
    const int c = blockIdx.x / C;
    const int rank = C == 1 ? 0 : int(cluster_rank());
    unsigned char *stages = smem_raw;
    T *xs = a.use_smem ? reinterpret_cast<T *>(smem_raw + kStages * kStageBytes) : nullptr;
    ring_init(&R);
    const int inst = a.dc.inst[c];
    double *vm = a.vm + (long long)c * nbus;
    double *va = a.va + (long long)c * nbus;
    double *cs = a.ef + (long long)c * 4 * nbus + 2 * nbus;
    double *sn = cs + nbus;
    const double *xg = a.xg + (long long)c * 2 * nbus;
    double *flag = a.bmax + (long long)c * 16 + 15;
    const T *F0 = static_cast<const T *>(a.F0) + (long long)inst * a.m0.stride;
    const T *F1 = static_cast<const T *>(a.F1) + (long long)inst * a.m1.stride;
    const int slice = (nbus + C - 1) / C;
    const int i0 = rank * slice, i1 = min(nbus, i0 + slice);
    int status = PF_ERR_NOT_CONVERGED;
    if (a.fs0[inst] != PF_OK) status = a.fs0[inst];
    else if (a.fs1[inst] != PF_OK) status = a.fs1[inst];
    int iters = 0;
    double mis = INFINITY;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        if (a.flat) {
            const int t = dn.btype[i];
            vm[i] = (t == PF_BUS_PQ) ? 1.0 : dn.vset[i];
            va[i] = (t == PF_BUS_SLACK) ? dn.va0[i] : 0.0;
        }
        sincos(va[i], &sn[i], &cs[i]);
    }
    cluster_sync<C>();
    if (status == PF_ERR_NOT_CONVERGED) {
        for (int it = 0; it < a.max_iter; it++) {
            mis = cluster_mismatch<C>(a, c, rank, 0, red);
            if (!isfinite(mis)) { status = PF_ERR_NONFINITE; break; }
            if (mis <= a.tol) { status = PF_OK; break; }
            if (rank == 0) {
                const bool ok = rank0_solve<T>(a, &R, stages, xs, a.m0, F0, c);
                if (threadIdx.x == 0) *flag = ok ? 0.0 : 1.0;
            }
            cluster_sync<C>();
            if (*flag != 0.0) { status = PF_ERR_TIMEOUT; break; }
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const int k = a.m0.new_of_bus[i];
                if (k >= 0) {
                    va[i] += xg[k];
                    sincos(va[i], &sn[i], &cs[i]);
                }
            }
            iters++;
            mis = cluster_mismatch<C>(a, c, rank, 1, red);
            if (!isfinite(mis)) { status = PF_ERR_NONFINITE; break; }
            if (mis <= a.tol) { status = PF_OK; break; }
            if (rank == 0) {
                const bool ok = rank0_solve<T>(a, &R, stages, xs, a.m1, F1, c);
                if (threadIdx.x == 0) *flag = ok ? 0.0 : 1.0;
            }
            cluster_sync<C>();
            if (*flag != 0.0) { status = PF_ERR_TIMEOUT; break; }
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const int k = a.m1.new_of_bus[i];
                if (k >= 0) vm[i] += xg[k];
            }
            iters++;
        }
        if (status == PF_ERR_NOT_CONVERGED) {
            mis = cluster_mismatch<C>(a, c, rank, 0, red);
            if (mis <= a.tol) status = PF_OK;
        }
    }
    if (rank == 0 && threadIdx.x == 0) {
        a.res[c].status = status;
        a.res[c].iters = iters;
        a.res[c].ir_steps = 0;
        a.res[c].pad = 0;
        a.res[c].max_mismatch = mis;
    }
    cluster_sync<C>();
}

int grid_for(long long total, int threads) {
    long long b = (total + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return int(b);
}

template <class T, int C>
cudaError_t launch_fdpf_t(const RunArgs &a, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_fdpf<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(a.dc.ncase) * C);
    cfg.blockDim = dim3(kRunThreads);
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
    const long long total = (long long)dc.ninst * (m.n + m.nnz);
    k_assemble_slots<<<grid_for(total, 256), 256, 0, s>>>(dn, dc, m, which, A);
    return cudaGetLastError();
}

cudaError_t launch_factor(const DevMat &m, int prec, const double *A, void *F, int ninst,
                          int *fstatus, cudaStream_t s) {
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

cudaError_t launch_solve(const DevMat &m, int prec, const void *F, const int *inst_of_case,
                         double *rhs, int ncase, void *gvec, int *status, size_t smem_optin,
                         cudaStream_t s) {
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
                                                            inst_of_case, rhs,
                                                            static_cast<double *>(gvec), use_smem,
                                                            status);
    } else {
        cudaFuncSetAttribute(k_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        k_solve<float><<<ncase, kSolveThreads, smem, s>>>(m, static_cast<const float *>(F),
                                                          inst_of_case, rhs,
                                                          static_cast<float *>(gvec), use_smem,
                                                          status);
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

// Cluster size of the power-flow kernel: a case spreads its nodal work over
// 16 (or 8) SMs when the batch is too small to fill the GPU with one block per
// case and such clusters can be resident; otherwise one block per case.
int fdpf_cluster_size(int ncase, int num_sms, int prec, size_t smem_optin, int nmax) {
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    size_t smem = size_t(kStages) * kStageBytes + elt * size_t(nmax);
    if (smem + 2048 > smem_optin) smem = size_t(kStages) * kStageBytes;
    for (int C : {16, 8}) {
        if (ncase * C > num_sms) continue;
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
        cudaError_t e;
        if (prec == PF_FP64) {
            auto *k = (C == 16) ? k_fdpf<double, 16> : k_fdpf<double, 8>;
            if (C == 16) cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            e = cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg);
        } else {
            auto *k = (C == 16) ? k_fdpf<float, 16> : k_fdpf<float, 8>;
            if (C == 16) cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            e = cudaOccupancyMaxActiveClusters(&nclusters, k, &cfg);
        }
        if (e == cudaSuccess && nclusters >= ncase) return C;
        cudaGetLastError();
    }
    return 1;
}

cudaError_t launch_fdpf(const DevNet &dn, const DevCases &dc, const DevMat *m, int prec,
                        const void *F0, const void *F1, const int *fstat0, const int *fstat1,
                        const pf_run_opts &o, double *vm, double *va, double *ef, double *xg,
                        double *bmax, pf_case_result *res, size_t smem_optin, int cluster,
                        cudaStream_t s) {
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
    if (!a.use_smem) smem = ring;
    if (prec == PF_FP64) {
        if (cluster >= 16) return launch_fdpf_t<double, 16>(a, smem, s);
        if (cluster >= 8) return launch_fdpf_t<double, 8>(a, smem, s);
        return launch_fdpf_t<double, 1>(a, smem, s);
    }
    if (cluster >= 16) return launch_fdpf_t<float, 16>(a, smem, s);
    if (cluster >= 8) return launch_fdpf_t<float, 8>(a, smem, s);
    return launch_fdpf_t<float, 1>(a, smem, s);
}

}  // namespace gbpf
