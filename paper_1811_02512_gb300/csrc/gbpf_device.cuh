// gbpf_device.cuh -- device helpers shared by the CUDA translation units of
// libgbpf: reductions, TMA bulk copies and mbarriers, cluster barriers, the
// TMA-staged level sweeps of the substitutions (Section III.C of arxiv
// 1811.02512) and the nodal injection (Section II.A).
#pragma once

#include <cfloat>
#include <cmath>
#include <cstdint>

#include "gbpf_internal.h"

namespace gbpf {
namespace {

constexpr int kFactorThreads = 512;
constexpr int kSolveThreads = 512;
constexpr int kRunThreads = 512;
constexpr int kStages = kRingStages;        // ring depth of the staged sweeps
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

// |x| as its IEEE-754 bit pattern: non-negative doubles order like their bit
// patterns read as unsigned integers, with every NaN above infinity, so a
// running maximum of these keys is the NaN-winning maximum of |x| and runs
// on the integer pipe instead of the (slow) FP64 one.
__device__ __forceinline__ unsigned long long abs_key(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
}

// Block-wide maximum of abs_key values; every thread receives the result.
// `red` is a 33-entry shared array.  Contains two __syncthreads.
__device__ unsigned long long block_max_key(unsigned long long v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long *r = reinterpret_cast<unsigned long long *>(red);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    if (lane == 0) r[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = (lane < int(blockDim.x >> 5)) ? r[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long u = __shfl_xor_sync(0xffffffffu, w, o);
            w = u > w ? u : w;
        }
        if (lane == 0) r[32] = w;
    }
    __syncthreads();
    return r[32];
}

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

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Barrier among the first `nthreads` threads of the block (named barrier 1)
// that ORs `pred` over them: every participant receives the same result, so
// a decision taken on it is uniform over the participants.
__device__ __forceinline__ bool consumer_vote_any(int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " barrier.cta.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"(uint32_t(pred)), "r"(nthreads)
        : "memory");
    return r != 0;
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

// Waits for phase `parity` of `bar`, giving up after `limit` polls, or
// earlier once *stop (optional) is non-zero.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned limit,
                                                  const volatile int *stop = nullptr) {
    for (unsigned i = 0; i < limit; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (stop && *stop) return false;
    }
    return false;
}

// Asks the L2 to fetch bytes [0, nbytes) of an array (rounded down to 16-byte
// multiples, within the allocation), in chunks of 32 KB spread over the
// calling threads: part (of nparts) is this thread's share.  A hint only:
// later loads of the range hit the L2 instead of waiting for DRAM.
__device__ __forceinline__ void l2_prefetch(const void *base, size_t nbytes, int part, int nparts) {
    constexpr size_t kChunk = 32768;
    const uintptr_t b0 = reinterpret_cast<uintptr_t>(base);
    const uintptr_t a0 = (b0 + 15) & ~uintptr_t(15);
    if (nbytes < (a0 - b0) + 16) return;
    const size_t usable = (nbytes - (a0 - b0)) & ~size_t(15);
    for (size_t off = size_t(part) * kChunk; off < usable; off += size_t(nparts) * kChunk) {
        const unsigned len = unsigned(usable - off < kChunk ? usable - off : kChunk);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0 + off), "r"(len) : "memory");
    }
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

// ------------------------------------------------------------ DSMEM access

__device__ __forceinline__ uint32_t cl_mapa(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}

__device__ __forceinline__ double ld_cl(uint32_t a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_cl_u64(uint32_t a) {
    unsigned long long v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ void st_cl(uint32_t a, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

__device__ __forceinline__ void st_cl(uint32_t a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

// Cluster barrier with release / acquire semantics at cluster scope: the
// shared-memory writes of every CTA before it are visible to every CTA
// after it.
__device__ __forceinline__ void cl_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The same for phases that exchange data through global memory as well:
// the release / acquire of the cluster barrier covers every state space
// (global stores before it are visible to loads after it in the cluster).
__device__ __forceinline__ void cl_barrier_global() { cl_barrier(); }

// ------------------------------------------------------------ staged sweeps

// Shared-memory ring of kStages stages; each stage holds one piece: row
// pointers, indices and values of a run of rows of one level.
struct Ring {
    uint64_t bar[kStages];   // full: the stage's copies have landed
    uint64_t ebar[kStages];  // empty: the consumers are done with the stage
    int hdr[kStages][20]; // r0, r1, e0, p_lo, i_lo, v_lo, idx off, val off, mode, run_end,
                          // diag off (-1: none), d_lo, level-pointer off, lp_lo, l0, l1, e1
    int err;              // set when a wait gave up
    unsigned gcount;      // pieces consumed so far (phase bookkeeping)
    // Self-test hooks of the give-up path (-1 = off; only the sweep self-test
    // sets them), in pieces counted since ring_init: the producer issues no
    // piece from number `stall_at` on, as if its copies never landed, and the
    // consumers do not release the stage of piece number `hold_at`, as if they
    // never finished with it.  Either makes a bounded wait of a sweep run out.
    int stall_at, hold_at;
};

__device__ void ring_init(Ring *R) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&R->bar[s], 1);
            mbar_init(&R->ebar[s], 1);
        }
        R->err = 0;
        R->gcount = 0;
        R->stall_at = -1;
        R->hold_at = -1;
        fence_mbar_init();
    }
    __syncthreads();
}

// Issues piece `pc` of a sweep over (ptr, idx, val) into stage `st`.  Values
// are NB x NB blocks (NB = 1: scalars) of type T; `dinv` (optional) holds the
// inverse diagonal blocks of the rows.  Called by one thread.  Ranges are
// widened to 16-byte boundaries; the arrays are padded so the widened ranges
// stay inside their allocations.
template <class T, int NB>
__device__ void ring_issue(Ring *R, unsigned char *stages, int st, const Piece &pc, const int *ptr,
                           const int *idx, const T *val, const T *dinv, const int *lvl_ptr) {
    constexpr int V = 16 / int(sizeof(T));
    constexpr int NB2 = NB * NB;
    const int p_lo = pc.r0 & ~3, p_hi = (pc.r1 + 1 + 3) & ~3;
    const int i_lo = pc.e0 & ~3, i_hi = (pc.e1 + 3) & ~3;
    const int v_lo = (pc.e0 * NB2) & ~(V - 1), v_hi = (pc.e1 * NB2 + V - 1) & ~(V - 1);
    const int d_lo = (pc.r0 * NB2) & ~(V - 1), d_hi = (pc.r1 * NB2 + V - 1) & ~(V - 1);
    const uint32_t pbytes = uint32_t(p_hi - p_lo) * 4u;
    const uint32_t ibytes = pc.e1 > pc.e0 ? uint32_t(i_hi - i_lo) * 4u : 0u;
    const uint32_t vbytes = (pc.e1 > pc.e0 && val) ? uint32_t(v_hi - v_lo) * uint32_t(sizeof(T)) : 0u;
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
    h[16] = pc.e1;
    unsigned char *dst = stages + size_t(st) * kStageBytes;
    fence_proxy_async();
    mbar_arrive_expect_tx(&R->bar[st], pbytes + ibytes + vbytes + dbytes + lbytes);
    tma_g2s(dst, ptr + p_lo, pbytes, &R->bar[st]);
    if (ibytes) tma_g2s(dst + ioff, idx + i_lo, ibytes, &R->bar[st]);
    if (vbytes) tma_g2s(dst + voff, val + v_lo, vbytes, &R->bar[st]);
    if (dbytes) tma_g2s(dst + doff, dinv + d_lo, dbytes, &R->bar[st]);
    if (lbytes) tma_g2s(dst + loff, lvl_ptr + lp_lo, lbytes, &R->bar[st]);
}

template <class X>
__device__ __forceinline__ X warp_sum(X v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Small fixed-size vector for the NB unknowns of one row.
template <class X, int NB>
struct Vec {
    X v[NB];
};

// y += B x for an NB x NB block B (row-major, TRANS: B^T).
template <class T, class X, int NB, bool TRANS>
__device__ __forceinline__ void blk_mac(Vec<X, NB> &y, const T *B, const X *x) {
#pragma unroll
    for (int i = 0; i < NB; i++)
#pragma unroll
        for (int j = 0; j < NB; j++) y.v[i] += X(B[TRANS ? j * NB + i : i * NB + j]) * x[j];
}

// Row r of a piece: x_r = (Dinv_r x_r when the piece carries the inverse
// diagonal) - sum over the entries (B_e or B_e^T) x_{idx_e}, over lanes
// [gl, len) with step gsz; the caller reduces `acc` over the lanes.
template <class T, class X, int NB, bool TRANS>
__device__ __forceinline__ void row_partial(Vec<X, NB> &acc, const int *P, const int *I, const T *Vv,
                                            X *x, int r, int p_lo, int i_lo, int v_lo, int gl,
                                            int gsz) {
    const int a = P[r - p_lo], b = P[r + 1 - p_lo];
    for (int e = a + gl; e < b; e += gsz)
        blk_mac<T, X, NB, TRANS>(acc, Vv + (e * NB * NB - v_lo), x + size_t(I[e - i_lo]) * NB);
}

template <class T, class X, int NB, bool TRANS>
__device__ __forceinline__ void row_finish(const Vec<X, NB> &acc, const T *Dv, int d_lo, X *x, int r) {
    X xr[NB], out[NB];
#pragma unroll
    for (int i = 0; i < NB; i++) xr[i] = x[size_t(r) * NB + i];
    if (Dv) {
        Vec<X, NB> t;
#pragma unroll
        for (int i = 0; i < NB; i++) t.v[i] = X(0);
        blk_mac<T, X, NB, TRANS>(t, Dv + (r * NB * NB - d_lo), xr);
#pragma unroll
        for (int i = 0; i < NB; i++) out[i] = t.v[i] - acc.v[i];
    } else {
#pragma unroll
        for (int i = 0; i < NB; i++) out[i] = xr[i] - acc.v[i];
    }
#pragma unroll
    for (int i = 0; i < NB; i++) x[size_t(r) * NB + i] = out[i];
}

// Rows of one staged piece.  mode 0: thread per row; mode 1: groups of 8
// lanes per row over all warps; mode 2: the calling warp alone walks the narrow levels
// l0..l1 of the piece (ascending forward, descending when the piece carries
// the diagonal, i.e. in the back substitution), split into groups of 32/R
// lanes for the R rows of each level.  Entries of a row are spread over the
// lanes of its warp or group and summed by shuffles.
template <class T, class X, int NB, bool TRANS>
__device__ __forceinline__ void piece_rows(const int *h, const unsigned char *base, X *x, int mode,
                                           int first, int stride) {
    const int *P = reinterpret_cast<const int *>(base);
    const int *I = reinterpret_cast<const int *>(base + h[6]);
    const T *Vv = reinterpret_cast<const T *>(base + h[7]);
    const T *Dv = h[10] >= 0 ? reinterpret_cast<const T *>(base + h[10]) : nullptr;
    const int r0 = h[0], r1 = h[1], p_lo = h[3], i_lo = h[4], v_lo = h[5], d_lo = h[11];
    const int lane = threadIdx.x & 31;
    if (mode == 4) {
        // scatter over the tail rows (NB = 1): slot rows [e0/32, e1/32) of the
        // tail levels r0..r1-1; a lane applies x_i -= l x_j for its own rows i
        // Within a level the sources are never targets, so a batch of slots
        // loads its indices, values and source entries first; a lane's slots
        // are sorted by target, so consecutive updates of one row accumulate
        // in a register and the row is read and written once per batch.
        const int k0 = h[2] >> 5, k1 = h[16] >> 5;
        X *xt = x + h[14];
        for (int lv = r0; lv < r1; lv++) {
            const int ka = max(P[lv - p_lo], k0), kb = min(P[lv + 1 - p_lo], k1);
            for (int k = ka; k < kb; k += 4) {
                int pk[4];
                X v[4], xs[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int sl = (k + u) * 32 + lane;
                    pk[u] = k + u < kb ? I[sl - i_lo] : -1;
                    v[u] = pk[u] >= 0 ? X(Vv[sl - v_lo]) : X(0);
                }
#pragma unroll
                for (int u = 0; u < 4; u++) xs[u] = pk[u] >= 0 ? xt[pk[u] >> 16] : X(0);
                int cur = -1;
                X acc = X(0);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    if (pk[u] < 0) continue;
                    const int tg = pk[u] & 0xffff;
                    if (tg != cur) {
                        if (cur >= 0) xt[cur] = acc;
                        cur = tg;
                        acc = xt[tg];
                    }
                    acc -= v[u] * xs[u];
                }
                if (cur >= 0) xt[cur] = acc;
            }
            __syncwarp();
        }
    } else if (mode == 0 || mode == 6) {
        for (int r = r0 + first; r < r1; r += stride) {
            Vec<X, NB> acc;
#pragma unroll
            for (int i = 0; i < NB; i++) acc.v[i] = X(0);
            row_partial<T, X, NB, TRANS>(acc, P, I, Vv, x, r, p_lo, i_lo, v_lo, 0, 1);
            row_finish<T, X, NB, TRANS>(acc, Dv, d_lo, x, r);
        }
    } else if (mode == 3) {
        // part [e0, e1) of row r0 on the calling warp; the diagonal is applied
        // by the part that starts the row
        const int e0 = h[2], e1 = h[16];
        Vec<X, NB> acc;
#pragma unroll
        for (int i = 0; i < NB; i++) acc.v[i] = X(0);
        for (int e = e0 + lane; e < e1; e += 32)
            blk_mac<T, X, NB, TRANS>(acc, Vv + (e * NB * NB - v_lo), x + size_t(I[e - i_lo]) * NB);
#pragma unroll
        for (int i = 0; i < NB; i++) acc.v[i] = warp_sum(acc.v[i]);
        if (lane == 0)
            row_finish<T, X, NB, TRANS>(acc, e0 == P[r0 - p_lo] ? Dv : nullptr, d_lo, x, r0);
    } else if (mode == 1 || mode == 5) {
        // groups of G lanes per row, 32 / G rows per warp and round: the rows
        // of these pieces are short (mode 1, G = 8) or of moderate length
        // (mode 5, G = 4), so a two- or three-step reduction suffices
        const int G = mode == 1 ? 8 : 4;
        const int grp = lane / G, gl = lane % G;
        for (int rb = r0 + first * (32 / G); rb < r1; rb += stride * (32 / G)) {
            const int r = rb + grp;
            Vec<X, NB> acc;
#pragma unroll
            for (int i = 0; i < NB; i++) acc.v[i] = X(0);
            if (r < r1) row_partial<T, X, NB, TRANS>(acc, P, I, Vv, x, r, p_lo, i_lo, v_lo, gl, G);
            for (int o = G >> 1; o > 0; o >>= 1)
#pragma unroll
                for (int i = 0; i < NB; i++) acc.v[i] += __shfl_xor_sync(0xffffffffu, acc.v[i], o);
            if (r < r1 && gl == 0) row_finish<T, X, NB, TRANS>(acc, Dv, d_lo, x, r);
        }
    } else {
        const int *LP = reinterpret_cast<const int *>(base + h[12]) - h[13];
        const int l0 = h[14], l1 = h[15];
        const bool down = Dv != nullptr;
        for (int li = 0; li <= l1 - l0; li++) {
            const int l = down ? l1 - li : l0 + li;
            const int lr0 = max(LP[l], r0), lr1 = min(LP[l + 1], r1);
            const int lrows = lr1 - lr0;
            const int gsz = lrows <= 1 ? 32 : lrows <= 2 ? 16 : lrows <= 4 ? 8 : lrows <= 8 ? 4 : 2;
            const int grp = lane / gsz, gl = lane % gsz;
            for (int i0 = 0; i0 < lrows; i0 += 32 / gsz) {
                const int i = i0 + grp;
                Vec<X, NB> acc;
#pragma unroll
                for (int k = 0; k < NB; k++) acc.v[k] = X(0);
                const int r = i < lrows ? lr0 + i : -1;
                if (r >= 0) row_partial<T, X, NB, TRANS>(acc, P, I, Vv, x, r, p_lo, i_lo, v_lo, gl, gsz);
                for (int o = gsz >> 1; o > 0; o >>= 1)
#pragma unroll
                    for (int k = 0; k < NB; k++) acc.v[k] += __shfl_xor_sync(0xffffffffu, acc.v[k], o);
                if (r >= 0 && gl == 0) row_finish<T, X, NB, TRANS>(acc, Dv, d_lo, x, r);
            }
            __syncwarp();
        }
    }
}

// Arrays staged for the pieces of one sweep: modes 0-3 read (ptr, idx, val,
// dinv, lvl_ptr); mode 4 the scatter schedule (ptr4 slot-row offsets, idx4
// slots, val4 slot values); mode 5 the tail rows' entries below the tail
// (ptr5, idx5, val5); mode 6 only the inverse diagonal (ptr6: zeros).
template <class T>
struct SweepSrc {
    const int *ptr, *idx;
    const T *val, *dinv;
    const int *lvl_ptr;
    const int *ptr4, *idx4;
    const T *val4;
    const int *ptr5, *idx5;
    const T *val5;
    const int *ptr6;
};

template <class T, int NB>
__device__ __forceinline__ void issue_piece(Ring *R, unsigned char *stages, int st, const Piece &pc,
                                            const SweepSrc<T> &S) {
    if (pc.mode == 4)
        ring_issue<T, NB>(R, stages, st, pc, S.ptr4, S.idx4, S.val4, nullptr, nullptr);
    else if (pc.mode == 5)
        ring_issue<T, NB>(R, stages, st, pc, S.ptr5, S.idx5, S.val5, nullptr, nullptr);
    else if (pc.mode == 6)
        ring_issue<T, NB>(R, stages, st, pc, S.ptr6, nullptr, nullptr, S.dinv, nullptr);
    else
        ring_issue<T, NB>(R, stages, st, pc, S.ptr, S.idx, S.val, S.dinv, S.lvl_ptr);
}

// One substitution sweep: for every piece in order, every row r of the piece
// gets x_r -= sum_e val_e x_{idx_e} (NB x NB blocks, optionally transposed,
// with the inverse diagonal applied first when given).  Pieces of the same
// level are independent.  The last warp of the block is the producer: it
// issues each piece's copies into the ring as soon as the consumers have
// released the stage's previous piece (an "empty" mbarrier per stage), so
// issuing is off the consumers' critical path.  The other warps consume:
// a block-wide piece is computed by all of them; a run of single-warp
// pieces (modes 2-4) is consumed by warp 0 alone, which releases each stage
// as it goes, while the other consumers go on to wait for the piece after
// the run.
//
// Giving up is collective.  Before each piece every consumer waits (bounded)
// for the piece's copies and reads the two header words that steer the
// control flow (mode, run end); then all consumers vote at one named barrier
// (consumer_vote_any) on whether anyone's wait gave up or the error flag is
// set.  On "stop" all of them leave at that same barrier, so none is left
// waiting at a later one, and a header is acted on only after the vote has
// confirmed that every consumer saw its copies land.  The vote is also the
// barrier after which a block-wide piece's stage is released.  Warp 0's
// decisions inside a run are taken by __any_sync over its lanes, and a run
// ends with a vote of its own before anyone waits for the next piece: a
// parity wait is only sound once the stage's previous phase (the piece four
// before) has completed, which only warp 0 has seen for the run's pieces.  After the
// sweep, if anything gave up, the producer waits for every copy it issued
// that may still be in flight (a copy must not outlive the block).  Returns
// false if a wait gave up (the same value in every thread).
template <class T, class X, int NB, bool TRANS>
__device__ bool staged_sweep(Ring *R, unsigned char *stages, const Piece *pieces, int np,
                             const SweepSrc<T> &S, X *x, unsigned spin) {
    const unsigned g0 = R->gcount;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int ncw = nwarps - 1, nct = ncw * 32;  // consumer warps / threads
    volatile int *err = &R->err;
    int issued = 0;  // producer lane 0: pieces whose copies were issued
    if (warp == ncw) {
        // producer: piece j goes into stage (g0 + j) mod kStages once the
        // consumers have released that stage's previous piece
        if (lane == 0) {
            const int stall = R->stall_at;
            for (int j = 0; j < np; j++) {
                const unsigned g = g0 + unsigned(j);
                if (stall >= 0 && g >= unsigned(stall)) break;  // self-test: these copies never come
                const int st = int(g % kStages);
                if (g >= unsigned(kStages) &&
                    !mbar_wait_bounded(&R->ebar[st], ((g / kStages) & 1u) ^ 1u, spin, err)) {
                    atomicExch(&R->err, 1);
                    break;
                }
                if (*err) break;
                issue_piece<T, NB>(R, stages, st, pieces[j], S);
                issued = j + 1;
            }
        }
        __syncwarp();
    } else {
        const int hold = R->hold_at;
        // wait for piece jx and peek at its control words (valid only when
        // the wait succeeded; used only after a vote confirmed that)
        auto wait_peek = [&](int jx, int &mode, int &run_end) {
            const unsigned g = g0 + unsigned(jx);
            const int st = int(g % kStages);
            const bool got = mbar_wait_bounded(&R->bar[st], (g / kStages) & 1u, spin, err);
            if (got) {
                mode = R->hdr[st][8];
                run_end = R->hdr[st][9];
            }
            return got;
        };
        int mode = 0, run_end = 0;
        bool stop = np > 0 ? consumer_vote_any(nct, !wait_peek(0, mode, run_end) || *err != 0) : false;
        int j = 0;
        while (!stop && j < np) {
            const int st = int((g0 + unsigned(j)) % kStages);
            const bool run = mode >= 2 && mode <= 4;
            const int jn = run ? run_end : j + 1;
            bool fail = false;
            if (run) {
                if (warp == 0) {
                    for (int jj = j; jj < jn; jj++) {
                        const unsigned gg = g0 + unsigned(jj);
                        const int s2 = int(gg % kStages);
                        if (jj > j) {
                            const bool got = mbar_wait_bounded(&R->bar[s2], (gg / kStages) & 1u, spin, err);
                            if (__any_sync(0xffffffffu, !got || *err != 0)) {
                                fail = true;
                                break;
                            }
                        }
                        piece_rows<T, X, NB, TRANS>(R->hdr[s2], stages + size_t(s2) * kStageBytes, x,
                                                    R->hdr[s2][8], 0, 1);
                        __syncwarp();
                        if (lane == 0 && int(gg) != hold) mbar_arrive(&R->ebar[s2]);
                    }
                    if (fail && lane == 0) atomicExch(&R->err, 1);
                }
                // the other consumers wait here for warp 0: only once the run's
                // pieces have landed may they wait for the piece after it (the
                // stage's previous phase must be complete, or the parity wait
                // could succeed on it)
                if (consumer_vote_any(nct, fail || *err != 0)) {
                    stop = true;
                    break;
                }
            } else {
                piece_rows<T, X, NB, TRANS>(R->hdr[st], stages + size_t(st) * kStageBytes, x, mode,
                                            (mode == 1 || mode == 5) ? warp : int(threadIdx.x),
                                            (mode == 1 || mode == 5) ? ncw : nct);
            }
            int nmode = 0, nrun = 0;
            const bool got = jn < np ? wait_peek(jn, nmode, nrun) : true;
            stop = consumer_vote_any(nct, !got || *err != 0);
            // every consumer is done with a block-wide piece: release its stage
            if (!run && !stop && threadIdx.x == 0 && int(g0 + unsigned(j)) != hold)
                mbar_arrive(&R->ebar[st]);
            mode = nmode;
            run_end = nrun;
            j = jn;
        }
        if (stop && threadIdx.x == 0) atomicExch(&R->err, 1);
    }
    __syncthreads();
    const bool ok = R->err == 0;
    if (!ok && warp == ncw && lane == 0) {
        // drain: the last issued piece of every stage may still be in flight
        const unsigned long_spin = spin > kDefaultSpin ? spin : kDefaultSpin;
        for (int q = (issued > kStages ? issued - kStages : 0); q < issued; q++) {
            const unsigned gq = g0 + unsigned(q);
            mbar_wait_bounded(&R->bar[gq % kStages], (gq / kStages) & 1u, long_spin);
        }
    }
    if (threadIdx.x == 0) R->gcount = g0 + unsigned(np);
    __syncthreads();
    return ok;
}

// The same sweep over pieces of modes 0-3 only.
template <class T, class X, int NB, bool TRANS>
__device__ bool staged_sweep(Ring *R, unsigned char *stages, const Piece *pieces, int np,
                             const int *ptr, const int *idx, const T *val, const T *dinv,
                             const int *lvl_ptr, X *x, unsigned spin) {
    const SweepSrc<T> S{ptr, idx, val, dinv, lvl_ptr, nullptr, nullptr, nullptr,
                        nullptr, nullptr, nullptr, nullptr};
    return staged_sweep<T, X, NB, TRANS>(R, stages, pieces, np, S, x, spin);
}

// The narrow top [t0, n) of a substitution through its partitioned inverse
// (tail form 3, see DevMat): on entry x[t0..n) holds c_T = b_T - L_TB z_B;
// z_T = W c_T, then x_T = W^T D_T^-1 z_T.  Each gather runs a thread per
// chunk of a row's entries into partial sums, then a thread per row adding
// its own term and its chunks' sums in chunk order (a fixed order of
// operations).  `scratch` (the staging ring, idle between the two sweeps)
// holds z_T and the partial sums; the producer's proxy fence before its next
// copy orders these writes before the ring is refilled.
template <class T, class X>
__device__ void tail_inverse_solve(const DevMat &m, const T *tw, const T *Dinv, X *x, unsigned char *scratch) {
    const int t0 = m.t0, nt = m.nt;
    T *z = reinterpret_cast<T *>(scratch);
    T *part = z + nt;
    for (int k = threadIdx.x; k < m.tw_nfc; k += blockDim.x) {
        const int2 c = m.twfc[k];
        T acc = T(0);
        for (int e = c.x; e < c.y; e++) acc = fma(tw[e], T(x[t0 + m.twfj[e]]), acc);
        part[k] = acc;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nt; r += blockDim.x) {
        T acc = T(x[t0 + r]);
        for (int k = m.twfr[r]; k < m.twfr[r + 1]; k++) acc += part[k];
        z[r] = acc;
    }
    __syncthreads();
    const T *twb = tw + m.tw_boff;
    for (int k = threadIdx.x; k < m.tw_nbc; k += blockDim.x) {
        const int2 c = m.twbc[k];
        T acc = T(0);
        for (int e = c.x; e < c.y; e++) acc = fma(twb[e], z[m.twbj[e]], acc);
        part[k] = acc;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nt; r += blockDim.x) {
        T acc = z[r] * Dinv[t0 + r];
        for (int k = m.twbr[r]; k < m.twbr[r + 1]; k++) acc += part[k];
        x[t0 + r] = X(acc);
    }
    __syncthreads();
}

// L D L^T x = x in place (level order): forward substitution over the rows
// of L (levels ascending), then back substitution over the columns of L
// (levels descending) with the normalisation y = z / d of Eq. 4 fused in as
// a multiplication by the stored inverse diagonal.
//
// With the gathered tail values tv of the instance (and a matrix with a
// scatter tail), the sweeps run the tail levels as a one-warp scatter: the
// forward sweep ends with the tail rows' entries below the tail and the
// forward scatter; the backward sweep starts with the tail rows' inverse
// diagonal and the backward scatter.  With the tail-inverse values tw as
// well (tail form 3), the top is instead two gathers through its partitioned
// inverse between the two sweeps (tail_inverse_solve).
template <class T, class X>
__device__ bool block_solve(Ring *R, unsigned char *stages, const DevMat &m, const T *F, X *x,
                            unsigned spin, const T *tv = nullptr, const T *tw = nullptr) {
    if (tv && tw && m.npf3 > 0) {
        // the narrow top through its partitioned inverse (tail form 3)
        const SweepSrc<T> Sf{m.Fp, m.Fc, F + m.offLr, nullptr, m.lvl_ptr, m.SKf, m.SIf, tv + m.tv_f,
                             m.PPp, m.PPc, tv + m.tv_p, m.ZP};
        if (!staged_sweep<T, X, 1, false>(R, stages, m.pf3, m.npf3, Sf, x, spin)) return false;
        tail_inverse_solve<T, X>(m, tw, F + m.offDi, x, stages);
        const SweepSrc<T> Sb{m.Cp, m.Cr, F + m.offLc, F + m.offDi, m.lvl_ptr, m.SKb, m.SIb,
                             tv + m.tv_b, nullptr, nullptr, nullptr, m.ZP};
        return staged_sweep<T, X, 1, false>(R, stages, m.pb3, m.npb3, Sb, x, spin);
    }
    if (tv && m.npf2 > 0) {
        const SweepSrc<T> Sf{m.Fp, m.Fc, F + m.offLr, nullptr, m.lvl_ptr, m.SKf, m.SIf, tv + m.tv_f,
                             m.PPp, m.PPc, tv + m.tv_p, m.ZP};
        if (!staged_sweep<T, X, 1, false>(R, stages, m.pf2, m.npf2, Sf, x, spin)) return false;
        const SweepSrc<T> Sb{m.Cp, m.Cr, F + m.offLc, F + m.offDi, m.lvl_ptr, m.SKb, m.SIb,
                             tv + m.tv_b, nullptr, nullptr, nullptr, m.ZP};
        return staged_sweep<T, X, 1, false>(R, stages, m.pb2, m.npb2, Sb, x, spin);
    }
    if (!staged_sweep<T, X, 1, false>(R, stages, m.pf, m.npf, m.Fp, m.Fc, F + m.offLr, nullptr,
                                      m.lvl_ptr, x, spin))
        return false;
    return staged_sweep<T, X, 1, false>(R, stages, m.pb, m.npb, m.Cp, m.Cr, F + m.offLc,
                                        F + m.offDi, m.lvl_ptr, x, spin);
}

// 1 / v for the pivots of the factorisations, whose reciprocals sit on the
// level chain: Newton's iteration for the reciprocal, r <- r + r (1 - v r)
// (each step squares the relative error), started from the correctly rounded
// FP32 reciprocal (relative error below 2^-24): two steps reach the FP64
// rounding level (within an ulp or two of the quotient; a self-test checks
// this against CUDA's division).  Outside [2^-99, 2^99) -- well inside the
// FP32 range -- or for a zero or non-finite v, the plain division.  The
// range is read from the exponent field with integer instructions: on GB300
// every FP64 instruction, a compare included, costs its warp about 64
// cycles, and this sits on the factorisations' level chain.
__device__ __forceinline__ double pivot_recip(double v) {
    const unsigned ex = (unsigned(__double2hiint(v)) >> 20) & 0x7ffu;  // biased exponent
    if (ex < 1023u - 99u || ex >= 1023u + 99u) return 1.0 / v;
    double r = double(__frcp_rn(float(v)));
    r = fma(r, fma(-v, r, 1.0), r);
    r = fma(r, fma(-v, r, 1.0), r);
    return r;
}
__device__ __forceinline__ float pivot_recip(float v) { return 1.0f / v; }

// sin and cos of a small angle (|x| <= kRotMax) from their Maclaurin series,
// truncated after the x^11 (sin) and x^12 (cos) terms in Horner form; for
// |x| <= 0.2 the first omitted terms are below 2e-19, far under one unit in
// the last place.  When every active lane of the warp has |x| <= 1e-3 (the
// steps of all but the first iterations) the series stop after x^5 and x^4:
// the omitted terms are then below 2e-22 relative (sin) and 1.4e-21
// absolute (cos), and each function costs two multiply-adds instead of
// six.  Used to rotate cached (cos theta, sin theta) by a Newton/FDPF angle
// step instead of re-evaluating both functions.
constexpr double kRotMax = 0.2;
constexpr double kRotShort = 1e-3;

__device__ __forceinline__ void small_sincos(double x, double *s, double *c) {
    const double x2 = x * x;
    if (__all_sync(__activemask(), fabs(x) <= kRotShort)) {  // one path per warp
        *s = x + x * x2 * (x2 * (1.0 / 120.0) - 1.0 / 6.0);
        *c = 1.0 + x2 * (x2 * (1.0 / 24.0) - 0.5);
        return;
    }
    const double ps = 1.0 / 39916800.0;   // 1/11!
    double t = -ps;
    t = t * x2 + 1.0 / 362880.0;          // 1/9!
    t = t * x2 - 1.0 / 5040.0;            // 1/7!
    t = t * x2 + 1.0 / 120.0;             // 1/5!
    t = t * x2 - 1.0 / 6.0;               // 1/3!
    *s = x + x * x2 * t;
    double u = 1.0 / 479001600.0;         // 1/12!
    u = u * x2 - 1.0 / 3628800.0;         // 1/10!
    u = u * x2 + 1.0 / 40320.0;           // 1/8!
    u = u * x2 - 1.0 / 720.0;             // 1/6!
    u = u * x2 + 1.0 / 24.0;              // 1/4!
    u = u * x2 - 0.5;                     // 1/2!
    *c = 1.0 + x2 * u;
}

// Current at bus i of one case: I_i = sum_k Y_ik V_k on the base admittance
// matrix, minus the terms of the case's outaged branch (if any) at its end
// buses; returns (Re I_i, Im I_i).  The injection is S_i = V_i conj(I_i):
// P_i = e_i Re I_i + f_i Im I_i, Q_i = f_i Re I_i - e_i Im I_i.  Each
// admittance entry costs four fused multiply-adds (GB300's FP64 rate makes
// this loop the throughput floor of batches).
__device__ __forceinline__ void bus_current(const DevNet &dn, int i, int outage,
                                            const double *e, const double *f, double &ir_out,
                                            double &ii_out) {
    double ir = 0.0, ii = 0.0;
    // four entries at a time: all their loads are issued before the first
    // multiply-add waits, so a row costs one memory latency per four entries
    // (the row's order of operations is the same as one at a time)
    const int pe = dn.rowptr[i + 1];
    for (int p = dn.rowptr[i]; p < pe; p += 4) {
        int k[4];
        double g[4], b[4], ek[4], fk[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            k[u] = p + u < pe ? dn.col[p + u] : i;
            g[u] = p + u < pe ? dn.G[p + u] : 0.0;
            b[u] = p + u < pe ? dn.B[p + u] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            ek[u] = e[k[u]];
            fk[u] = f[k[u]];
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (p + u >= pe) break;
            ir = fma(g[u], ek[u], ir);
            ir = fma(-b[u], fk[u], ir);
            ii = fma(g[u], fk[u], ii);
            ii = fma(b[u], ek[u], ii);
        }
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
    ir_out = ir;
    ii_out = ii;
}

// Injection at bus i of one case, S_i = V_i conj(I_i) as (P, Q).
__device__ __forceinline__ void bus_injection(const DevNet &dn, int i, int outage,
                                              const double *e, const double *f, double &P,
                                              double &Q) {
    double ir, ii;
    bus_current(dn, i, outage, e, f, ir, ii);
    P = e[i] * ir + f[i] * ii;
    Q = f[i] * ir - e[i] * ii;
}

}  // namespace
}  // namespace gbpf
