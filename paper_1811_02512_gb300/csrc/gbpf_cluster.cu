// gbpf_cluster.cu -- single-case fast-decoupled power flow with the
// substitutions spread over a thread-block cluster (sm_103a).
//
// One case runs on the C = 16 CTAs of a cluster, one per SM.  The nodal
// mismatch is split by bus slices as in k_fdpf (Section II.A).  The
// substitutions of Section III.C are split by rows: every row (column) of
// the factor has an owner CTA, which keeps that row's entries of L (and of
// the tail inverse below) resident in its shared memory for the whole
// launch, and holds the row's entry of the solution vector.
//
// The elimination forest is cut into a top set T (closed under taking
// parents; it holds the narrow top of the tree, a long run of levels with
// at most 16 rows each, 118 levels of B' at 10,000 buses) and the subtrees
// below it.  Every subtree belongs wholly to one CTA, so a level of it (the
// paper's hierarchical parallelism, Section II.B) reads only the CTA's own
// words and ends with the CTA's own barrier.  T is solved with the explicit
// inverse W = L_TT^-1 of its diagonal block of L (a partitioned inverse of
// the factor): with L = [[L_BB, 0], [L_TB, L_TT]],
//   forward   c_T = b_T - L_TB z_B,  z_T = W c_T,
//   backward  x_T = W^T D_T^-1 z_T,  then the subtrees' levels as usual,
// three cluster-wide steps whatever T's height, each reading other CTAs'
// words over the cluster's distributed shared memory and ending with a
// cluster barrier.  W has a nonzero (i, j) exactly when i is an ancestor of
// j in the elimination tree; it is formed after every factorisation by
// k_tail_inverse (a warp per column of T, right-looking along the column's
// ancestor path: w_i -= L_ik w_k), and gathered with the factor's values
// into the CTAs' packed value arrays by k_cl_values.
//
// A case the fast decoupled iteration leaves unconverged can fall back to
// Newton-Raphson (Section III) in the same launch: the cluster then reuses
// its shared memory for the Newton-Raphson staging ring and factor scratch
// (gbpf_nr.cuh).
#include "gbpf_nr.cuh"

namespace gbpf {

namespace {

constexpr int kClThreads = 512;

// ------------------------------------------------------------ tail inverse

// W = L_TT^-1 of the top set T of one matrix: W(it, jt) = Wd[it * nt + jt]
// (T-relative indices), written only where it is structurally nonzero (it
// an ancestor of, or equal to, jt).  One warp per column jt solves
// L_TT w = e_jt right-looking along jt's ancestor path: at path node k
// (ascending; tpar: parent, -1 at a root) w_k is final, and every entry
// L(i, k) of column k -- all on the path, since its rows are ancestors of k
// -- gives w_i -= L(i, k) w_k, one lane per entry (distinct rows, so no
// conflict).  The path's values live in shared memory by distance from jt
// (depth[jt] - depth[k]); the columns of L_TT (tcp, the depth of each
// entry's row in tcdep, its factor position in tcpos) are staged into shared
// memory first.  The order of operations is fixed.
template <class T>
__global__ void __launch_bounds__(kTailInvWarps * 32) k_tail_inverse(const ClMat m, const T *F, double *Wd) {
    extern __shared__ __align__(16) unsigned char tsm[];
    const int nt = m.nt, ne = m.ntail_e, D = m.tdepth_max;
    double *Lv = reinterpret_cast<double *>(tsm);
    double *wp = Lv + ne;                                   // [kTailInvWarps][D]
    int *Ld = reinterpret_cast<int *>(wp + kTailInvWarps * D);
    int *cp = Ld + ne;                                      // [nt + 1]
    int *dep = cp + nt + 1, *par = dep + nt;
    // the top's entries gathered from the factor, eight per thread in
    // flight (the positions first, then the values): the gather is most of
    // this kernel's time
    const int bd = int(blockDim.x);
    for (int q0 = threadIdx.x; q0 < ne; q0 += 8 * bd) {
        int pos[8];
        T val[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int q = q0 + u * bd;
            pos[u] = q < ne ? m.tcpos[q] : 0;
            if (q < ne) Ld[q] = m.tcdep[q];
        }
#pragma unroll
        for (int u = 0; u < 8; u++) val[u] = q0 + u * bd < ne ? F[pos[u]] : T(0);
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (q0 + u * bd < ne) Lv[q0 + u * bd] = double(val[u]);
    }
    for (int i = threadIdx.x; i <= nt; i += blockDim.x) cp[i] = m.tcp[i];
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        dep[i] = m.tdepth[i];
        par[i] = m.tpar[i];
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *w = wp + warp * D;
    for (int i = lane; i < D; i += 32) w[i] = 0.0;
    __syncthreads();
    const int jt = blockIdx.x * kTailInvWarps + warp;
    if (jt >= nt) return;
    const int dj = dep[jt];
    if (lane == 0) w[0] = 1.0;
    for (int k = jt; k >= 0; k = par[k]) {
        __syncwarp();
        const double wk = w[dj - dep[k]];
        if (lane == 0) Wd[(long long)k * nt + jt] = wk;
        for (int q = cp[k] + lane; q < cp[k + 1]; q += 32) {
            const int pos = dj - Ld[q];
            w[pos] = fma(-Lv[q], wk, w[pos]);
        }
    }
}

// Tail-inverse values of instance 0 (tail form 3 of the block engine):
// forward entries W(i, j), backward entries W(j, i) / D(j), from the dense W.
template <class T>
__global__ void k_tw_values(const DevMat m, const double *Wd, const T *F, T *TW) {
    const int tot = m.tw_nfe + m.tw_nbe;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
        if (e < m.tw_nfe) {
            TW[e] = T(Wd[m.twfs[e]]);
        } else {
            const int b = e - m.tw_nfe;
            TW[m.tw_boff + b] = T(Wd[m.twbs[b]] * double(F[m.offDi + m.twbd[b]]));
        }
    }
}

// Packed values of the CTAs' programs (blockIdx.y = matrix): per slot
// {kind, a, b}: 0 the factor value F[a]; 1 the negated tail-inverse entry
// -Wd[a] (forward tail step); 2 -Wd[a] * F[b] (backward tail step, the
// inverse diagonal folded in); 3 -GV[a], 4 -GV[a] * F[b] and 5 GV[a] (the
// grouped subtree steps: an entry of a group's inverse, the same with the
// inverse diagonal folded in, a combined entry).
__global__ void k_cl_values(const ClMat m0, const ClMat m1, const double *F0, const double *F1,
                            const double *W0, const double *W1) {
    const ClMat &m = blockIdx.y ? m1 : m0;
    const double *F = blockIdx.y ? F1 : F0;
    const double *Wd = blockIdx.y ? W1 : W0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < m.nval; s += gridDim.x * blockDim.x) {
        const int4 src = m.vsrc[s];
        double v;
        switch (src.x) {
            case 0: v = F[src.y]; break;
            case 1: v = -Wd[src.y]; break;
            case 2: v = -Wd[src.y] * F[src.z]; break;
            case 3: v = -m.gv[src.y]; break;
            case 4: v = -m.gv[src.y] * F[src.z]; break;
            default: v = m.gv[src.y]; break;
        }
        m.vals[s] = v;
    }
}

// Inverses of the subtree groups' blocks of L (blockIdx.y = matrix): one
// thread per inverse column j solves L_GG w = e_j along j's path to the top
// of its group, right-looking (w_q -= L(path[q], path[p]) w_p in the order
// of the update list), and writes W(path[q], j), q >= 1.
__global__ void k_cl_group_w(const ClMat m0, const ClMat m1, const double *F0, const double *F1) {
    const ClMat &m = blockIdx.y ? m1 : m0;
    const double *F = blockIdx.y ? F1 : F0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m.n_gwcol; c += gridDim.x * blockDim.x) {
        const int4 col = m.gw_col[c];
        double w[kClGroupMax];
        w[0] = 1.0;
#pragma unroll
        for (int q = 1; q < kClGroupMax; q++) w[q] = 0.0;
        for (int u = col.x; u < col.y; u++) {
            const int4 up = m.gw_upd[u];
            w[up.y] = fma(-F[up.z], w[up.x], w[up.y]);
        }
        for (int q = 1; q < col.w; q++) m.gv[col.z + q - 1] = w[q];
    }
}

// Combined entries of the grouped steps (blockIdx.y = matrix): the sum, in
// list order, of W(.) L(.) over the entry's terms (W = 1 for the identity).
__global__ void k_cl_group_m(const ClMat m0, const ClMat m1, const double *F0, const double *F1) {
    const ClMat &m = blockIdx.y ? m1 : m0;
    const double *F = blockIdx.y ? F1 : F0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m.n_gm; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int t = m.gm_ptr[e]; t < m.gm_ptr[e + 1]; t++) {
            const int2 tm = m.gm_term[t];
            const double w = tm.x < 0 ? 1.0 : m.gv[tm.x];
            s = fma(w, F[tm.y], s);
        }
        m.gv[m.n_gw + e] = s;
    }
}

// ------------------------------------------------------------ run kernel

struct ClRun {
    DevNet dn;
    DevCases dc;
    ClMat m[2];
    const int *fs0, *fs1;
    double tol;
    int max_iter;
    int flat;
    double *vm, *va;
    double *ef;    // [4 nbus]: e, f, cos(theta), sin(theta)
    double *iv;    // [nbus]: 1 / V
    double *bmax;  // [16]: per-CTA mismatch maxima
    pf_case_result *res;
    // FDPF -> NR fallback (Section III): an unconverged or non-finite end
    // restarts the case from a flat start under Newton-Raphson (nr) on the
    // same cluster, its shared memory reused for the staging ring and the
    // factor scratch; the result then reports method PF_NR
    int fallback;
    NrArgs nr;
};

// Shared-memory program of one matrix in one CTA (byte offsets of the
// regions are the same in every CTA, so a slot's address in another CTA is
// that CTA's base plus the same offset).
struct ClSmem {
    double *X;        // vector region
    int4 *tasks;      // {out, in, diag value or -1, first entry}, one sentinel
    int4 *steps;      // {first task, end task, lanes per task, 0}
    uint32_t *addr;   // entry sources as shared::cluster addresses
    double *vals;     // entry values, then the diagonal values
};

// One step of a sweep in this CTA: for each task t of the step,
// X[out] = (diag ? vals[diag] X[in] : X[in]) - sum_e vals[e] X(addr[e]),
// with G lanes per task (up to four entries per lane loaded at once and
// summed on one chain -- a warp's FP64 instructions do not overlap on
// GB300, so split chains would only add the combining ones -- the lanes'
// partial sums shuffle-reduced in lane order: the order of operations is
// fixed).  Warps without a task skip the step: on GB300 the FP64 pipe
// (about 1.7 FMA per cycle per SM) is shared by all warps, so idle
// arithmetic would delay the busy ones.
__device__ __forceinline__ void cl_step(const ClSmem &S, int4 si) {
    const int G = si.z;
    if (G == 1) {
        // one thread per task (most subtree levels): exactly one multiply-add
        // per entry, on one chain
        for (int t = si.x + int(threadIdx.x); t < si.y; t += kClThreads) {
            const int4 tk = S.tasks[t];
            const int e1 = S.tasks[t + 1].w;
            const double b = S.X[tk.y];
            const double dv = tk.z >= 0 ? S.vals[tk.z] : 1.0;
            double acc = 0.0;
            int e = tk.w;
            for (; e + 4 <= e1; e += 4) {
                const uint32_t p0 = S.addr[e], p1 = S.addr[e + 1], p2 = S.addr[e + 2], p3 = S.addr[e + 3];
                const double v0 = S.vals[e], v1 = S.vals[e + 1], v2 = S.vals[e + 2], v3 = S.vals[e + 3];
                const double x0 = ld_cl(p0), x1 = ld_cl(p1), x2 = ld_cl(p2), x3 = ld_cl(p3);
                acc = fma(v0, x0, acc);
                acc = fma(v1, x1, acc);
                acc = fma(v2, x2, acc);
                acc = fma(v3, x3, acc);
            }
            const int r = e1 - e;  // 0 to 3 entries left
            if (r > 0) {
                const uint32_t p0 = S.addr[e], p1 = S.addr[r > 1 ? e + 1 : e], p2 = S.addr[r > 2 ? e + 2 : e];
                const double v0 = S.vals[e], v1 = S.vals[r > 1 ? e + 1 : e], v2 = S.vals[r > 2 ? e + 2 : e];
                const double x0 = ld_cl(p0), x1 = ld_cl(p1), x2 = ld_cl(p2);
                acc = fma(v0, x0, acc);
                if (r > 1) acc = fma(v1, x1, acc);
                if (r > 2) acc = fma(v2, x2, acc);
            }
            S.X[tk.x] = fma(dv, b, -acc);
        }
        return;
    }
    const int per_warp = 32 / G;  // tasks per warp and round
    const int warp = int(threadIdx.x) >> 5, lane = int(threadIdx.x) & 31;
    const int grp = lane / G, gl = lane % G;
    for (int tb = si.x + warp * per_warp; tb < si.y; tb += (kClThreads / 32) * per_warp) {
        const int t = tb + grp;
        const bool act = t < si.y;
        double acc = 0.0, b = 0.0, dv = 1.0;
        int4 tk = make_int4(0, 0, -1, 0);
        if (act) {
            tk = S.tasks[t];
            const int e1 = S.tasks[t + 1].w;
            // every load that does not depend on the entries first: the task's
            // own word and diagonal value, then four entries' sources and
            // values, then their words, then the multiply-adds
            b = S.X[tk.y];
            if (tk.z >= 0) dv = S.vals[tk.z];
            for (int e = tk.w + gl; e < e1; e += 4 * G) {
                uint32_t p[4];
                double v[4], x[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const bool in = e + u * G < e1;
                    p[u] = in ? S.addr[e + u * G] : 0u;
                    v[u] = in ? S.vals[e + u * G] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 4; u++) x[u] = e + u * G < e1 ? ld_cl(p[u]) : 0.0;
                acc = fma(v[0], x[0], acc);
                if (e + G < e1) acc = fma(v[1], x[1], acc);
                if (e + 2 * G < e1) acc = fma(v[2], x[2], acc);
                if (e + 3 * G < e1) acc = fma(v[3], x[3], acc);
            }
        }
        for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (act && gl == 0) S.X[tk.x] = fma(dv, b, -acc);
    }
}

// Mismatch of one half-iteration (as k_fdpf's cluster_mismatch): the CTA's
// bus slice forms e + jf, then (after a cluster barrier) the currents of its
// rows; dP/V (which = 0) or dQ/V (which = 1) goes straight into the owner's
// vector slot of the matrix (rhsref: owner << 16 | word, -1 for a bus
// outside the matrix).  Returns the cluster maximum of the half-iteration's
// part (full: of both parts).  ef_ready: the slice's e + jf were already
// written with the state (by the update that produced it).
template <int C>
__device__ double cl_mismatch(const ClRun &a, int rank, int which, const uint32_t *xbase, double *red,
                              unsigned long long *mkey, const uint32_t *kbase, bool full, bool ef_ready) {
    const DevNet &dn = a.dn;
    const int nbus = dn.nbus;
    const int slice = (nbus + C - 1) / C;
    const int i0 = rank * slice, i1 = min(nbus, i0 + slice);
    double *e = a.ef;
    double *f = e + nbus;
    const double *cs = e + 2 * nbus;
    const double *sn = e + 3 * nbus;
    if (!ef_ready)
        for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            e[i] = a.vm[i] * cs[i];
            f[i] = a.vm[i] * sn[i];
        }
    cl_barrier_global();
    const int *rhsref = a.m[which].rhsref;
    const bool wantP = full || which == 0, wantQ = full || which == 1;
    unsigned long long mx = 0;
    for (int q = i0 + threadIdx.x; q < i1; q += blockDim.x) {
        const int i = C == kClCtas ? dn.mis_ord_cl[q] : q;  // a warp's rows of one length
        double ir, ii;
        bus_current(dn, i, -1, e, f, ir, ii);
        const int t = dn.btype[i];
        double dP = 0.0, dQ = 0.0;
        if (wantP && t != PF_BUS_SLACK) dP = a.dc.Psp[i] - (e[i] * ir + f[i] * ii);
        if (wantQ && t == PF_BUS_PQ) dQ = a.dc.Qsp[i] - (f[i] * ir - e[i] * ii);
        const unsigned long long kp = abs_key(dP), kq = abs_key(dQ);
        mx = kp > mx ? kp : mx;
        mx = kq > mx ? kq : mx;
        const int r = rhsref[i];
        if (r >= 0) st_cl(xbase[which * C + (r >> 16)] + 8u * unsigned(r & 0xffff), (which == 0 ? dP : dQ) * a.iv[i]);
    }
    mx = block_max_key(mx, red);
    // the CTAs' maxima are exchanged as integer keys through distributed
    // shared memory: slot `which` of each CTA's mkey
    if (threadIdx.x == 0) mkey[which] = mx;
    cl_barrier();
    unsigned long long k = 0;
    if (threadIdx.x < C) k = ld_cl_u64(kbase[threadIdx.x] + 8u * unsigned(which));
    for (int o = C / 2; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, k, o);
        k = u > k ? u : k;
    }
    k = __shfl_sync(0xffffffffu, k, 0);
    if ((threadIdx.x >> 5) == 0 && (threadIdx.x & 31) == 0) red[32] = __longlong_as_double(static_cast<long long>(k));
    __syncthreads();
    return red[32];
}

template <int C>
__global__ void __launch_bounds__(kClThreads, 1) k_fdpf_cl(const __grid_constant__ ClRun a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[33];
    __shared__ Ring R;  // the fallback's staging ring
    __shared__ uint32_t xbase[2 * C];  // vector region of matrix m in CTA r: xbase[m * C + r]
    __shared__ int nsteps[2];
    __shared__ unsigned long long mkey[2];  // this CTA's mismatch maximum (key) per half-iteration kind
    __shared__ uint32_t kbase[C];           // mkey of CTA r
    const int rank = int(cluster_rank());
    const DevNet &dn = a.dn;
    const int nbus = dn.nbus;
    // the CTA's programs into shared memory (same layout in every CTA)
    ClSmem S[2];
    for (int w = 0; w < 2; w++) {
        const ClMat &m = a.m[w];
        S[w].X = reinterpret_cast<double *>(smem_raw + m.so_x);
        S[w].tasks = reinterpret_cast<int4 *>(smem_raw + m.so_tasks);
        S[w].steps = reinterpret_cast<int4 *>(smem_raw + m.so_steps);
        S[w].addr = reinterpret_cast<uint32_t *>(smem_raw + m.so_addr);
        S[w].vals = reinterpret_cast<double *>(smem_raw + m.so_vals);
        if (threadIdx.x < C)
            xbase[w * C + threadIdx.x] = cl_mapa(smem_u32(smem_raw + m.so_x), threadIdx.x);
    }
    if (threadIdx.x < C) kbase[threadIdx.x] = cl_mapa(smem_u32(mkey), threadIdx.x);
    {  // the admittance matrix is read every half-iteration: start it towards the L2
        const int part = rank * kClThreads + int(threadIdx.x), parts = C * kClThreads;
        l2_prefetch(dn.col, sizeof(int) * size_t(dn.nnz), part, parts);
        l2_prefetch(dn.G, sizeof(double) * size_t(dn.nnz), part, parts);
        l2_prefetch(dn.B, sizeof(double) * size_t(dn.nnz), part, parts);
    }
    __syncthreads();
    for (int w = 0; w < 2; w++) {
        const ClMat &m = a.m[w];
        const int tb = m.tptr[rank], te = m.tptr[rank + 1];
        for (int t = threadIdx.x; t < te - tb; t += blockDim.x) S[w].tasks[t] = m.tasks[tb + t];
        const int sb = m.sptr[rank], se = m.sptr[rank + 1];
        for (int s = threadIdx.x; s < se - sb; s += blockDim.x) S[w].steps[s] = m.steps[sb + s];
        if (threadIdx.x == 0) nsteps[w] = se - sb;
        const int eb = m.eptr[rank], ee = m.eptr[rank + 1];
        for (int e = threadIdx.x; e < ee - eb; e += blockDim.x) {
            const int r = m.refs[eb + e];
            S[w].addr[e] = xbase[w * C + (r >> 16)] + 8u * unsigned(r & 0xffff);
        }
        const int vb = m.vptr[rank], ve = m.vptr[rank + 1];
        for (int v = threadIdx.x; v < ve - vb; v += blockDim.x) S[w].vals[v] = m.vals[vb + v];
    }
    if (a.fallback) ring_init(&R);
    // every CTA of the cluster has started (its shared memory exists) before
    // anyone writes to it
    cl_barrier();
    const int slice = (nbus + C - 1) / C;
    const int i0 = rank * slice, i1 = min(nbus, i0 + slice);
    double *vm = a.vm, *va = a.va, *iv = a.iv;
    double *ef = a.ef;  // e, f, then cos and sin of the angles
    double *cs = a.ef + 2 * nbus, *sn = cs + nbus;
    int status = PF_ERR_NOT_CONVERGED;
    if (a.fs0[0] != PF_OK) status = a.fs0[0];
    else if (a.fs1[0] != PF_OK) status = a.fs1[0];
    int iters = 0;
    double mis = INFINITY;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        if (a.flat) {
            const int t = dn.btype[i];
            vm[i] = (t == PF_BUS_PQ) ? 1.0 : dn.vset[i];
            va[i] = (t == PF_BUS_SLACK) ? dn.va0[i] : 0.0;
        }
        sincos(va[i], &sn[i], &cs[i]);
        iv[i] = 1.0 / vm[i];
        ef[i] = vm[i] * cs[i];
        ef[nbus + i] = vm[i] * sn[i];
    }
    // e + jf of every bus is written where the state changes (here, and in
    // the updates below), so the mismatch needs no pass of its own
    bool rotated = false;
    auto exact_check = [&](int which) {
        if (rotated)
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                sincos(va[i], &sn[i], &cs[i]);
                ef[i] = vm[i] * cs[i];
                ef[nbus + i] = vm[i] * sn[i];
            }
        rotated = false;
        return cl_mismatch<C>(a, rank, which, xbase, red, mkey, kbase, true, true);
    };
    // a step is followed by a cluster barrier (it read or feeds other CTAs'
    // words) or by the CTA's own barrier (a level of its own subtrees); every
    // CTA has the same number of cluster barriers
    auto solve = [&](int w) {
        const int ns = nsteps[w];
        for (int s = 0; s < ns; s++) {
            const int4 si = S[w].steps[s];
            cl_step(S[w], si);
            if (si.w) cl_barrier();
            else __syncthreads();
        }
    };
    // x of bus i after a solve of matrix w (owner << 16 | word, -1: none)
    auto xval = [&](int w, int i) {
        const int r = a.m[w].xref[i];
        return r >= 0 ? ld_cl(xbase[w * C + (r >> 16)] + 8u * unsigned(r & 0xffff)) : 0.0;
    };
    if (status == PF_ERR_NOT_CONVERGED) {
        for (int it = 0; it < a.max_iter; it++) {
            mis = cl_mismatch<C>(a, rank, 0, xbase, red, mkey, kbase, false, true);
            if (mis <= a.tol) mis = exact_check(0);
            if (!isfinite(mis)) { status = PF_ERR_NONFINITE; break; }
            if (mis <= a.tol) { status = PF_OK; break; }
            solve(0);
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                if (a.m[0].xref[i] < 0) continue;
                const double d = xval(0, i);
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
                ef[i] = vm[i] * cs[i];
                ef[nbus + i] = vm[i] * sn[i];
            }
            rotated = true;
            iters++;
            mis = cl_mismatch<C>(a, rank, 1, xbase, red, mkey, kbase, false, true);
            if (mis <= a.tol) mis = exact_check(1);
            if (!isfinite(mis)) { status = PF_ERR_NONFINITE; break; }
            if (mis <= a.tol) { status = PF_OK; break; }
            solve(1);
            for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                if (a.m[1].xref[i] < 0) continue;
                vm[i] += xval(1, i);
                iv[i] = 1.0 / vm[i];
                ef[i] = vm[i] * cs[i];
                ef[nbus + i] = vm[i] * sn[i];
            }
            iters++;
        }
        if (status == PF_ERR_NOT_CONVERGED) {
            mis = exact_check(0);
            if (mis <= a.tol) status = PF_OK;
        }
    }
    if (a.fallback && (status == PF_ERR_NOT_CONVERGED || status == PF_ERR_NONFINITE)) {
        cl_barrier();  // no CTA still reads or writes another's programs
        nr_fallback<double, C>(a.nr, 0, rank, smem_raw, red, &R);  // writes the case's result
        return;
    }
    if (rank == 0 && threadIdx.x == 0) {
        a.res[0].status = status;
        a.res[0].iters = iters;
        a.res[0].ir_steps = 0;
        a.res[0].method = PF_FDPF;
        a.res[0].max_mismatch = mis;
    }
    // no CTA leaves while another may still read its shared memory
    cl_barrier();
}

}  // namespace

// ------------------------------------------------------------ launchers

size_t tail_inverse_smem(int nt, int ne, int depth_max) {
    return sizeof(double) * (size_t(ne) + size_t(kTailInvWarps) * size_t(depth_max)) +
           sizeof(int) * (size_t(ne) + 3 * size_t(nt) + 1);
}

cudaError_t launch_tail_w(const DevMat &m, int prec, const void *F, double *Wd, void *TW, cudaStream_t s) {
    if (m.npf3 <= 0 || m.tw_ne <= 0) return cudaSuccess;
    ClMat t;  // the top's structure in the form k_tail_inverse reads
    t.nt = m.nt;
    t.ntail_e = m.tw_ne;
    t.tdepth_max = m.tw_depmax;
    t.tpar = m.twpar;
    t.tcp = m.twcp;
    t.tcdep = m.twcdep;
    t.tcpos = m.twcpos;
    t.tdepth = m.twdep;
    const size_t smem = tail_inverse_smem(t.nt, t.ntail_e, t.tdepth_max);
    const dim3 grid((t.nt + kTailInvWarps - 1) / kTailInvWarps);
    const int tot = m.tw_nfe + m.tw_nbe;
    const int vb = (tot + 255) / 256 < 1024 ? (tot + 255) / 256 : 1024;
    cudaError_t e;
    if (prec == PF_FP64) {
        e = cudaFuncSetAttribute(k_tail_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        k_tail_inverse<double><<<grid, kTailInvWarps * 32, smem, s>>>(t, static_cast<const double *>(F), Wd);
        k_tw_values<double><<<vb, 256, 0, s>>>(m, Wd, static_cast<const double *>(F), static_cast<double *>(TW));
    } else {
        e = cudaFuncSetAttribute(k_tail_inverse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        k_tail_inverse<float><<<grid, kTailInvWarps * 32, smem, s>>>(t, static_cast<const float *>(F), Wd);
        k_tw_values<float><<<vb, 256, 0, s>>>(m, Wd, static_cast<const float *>(F), static_cast<float *>(TW));
    }
    return cudaGetLastError();
}

cudaError_t launch_cl_inverse(const ClMat &m, const double *F, double *W, cudaStream_t s) {
    if (m.nt == 0) return cudaSuccess;
    const size_t smem = tail_inverse_smem(m.nt, m.ntail_e, m.tdepth_max);
    cudaError_t e = cudaFuncSetAttribute(k_tail_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    k_tail_inverse<double><<<(m.nt + kTailInvWarps - 1) / kTailInvWarps, kTailInvWarps * 32, smem, s>>>(m, F, W);
    return cudaGetLastError();
}

cudaError_t launch_cl_prepare(const ClMat &m0, const ClMat &m1, const double *F0, const double *F1,
                              double *W0, double *W1, cudaStream_t s) {
    const int nc = m0.n_gwcol > m1.n_gwcol ? m0.n_gwcol : m1.n_gwcol;
    if (nc > 0) k_cl_group_w<<<dim3(unsigned((nc + 255) / 256), 2), 256, 0, s>>>(m0, m1, F0, F1);
    const int nm = m0.n_gm > m1.n_gm ? m0.n_gm : m1.n_gm;
    if (nm > 0) k_cl_group_m<<<dim3(unsigned((nm + 255) / 256), 2), 256, 0, s>>>(m0, m1, F0, F1);
    const int nv = m0.nval > m1.nval ? m0.nval : m1.nval;
    k_cl_values<<<dim3(unsigned((nv + 255) / 256), 2), 256, 0, s>>>(m0, m1, F0, F1, W0, W1);
    return cudaGetLastError();
}

cudaError_t launch_fdpf_cl(const DevNet &dn, const DevCases &dc, const ClMat &m0, const ClMat &m1,
                           const int *fs0, const int *fs1, const pf_run_opts &o, double *vm, double *va,
                           double *ef, double *iv, double *bmax, pf_case_result *res, size_t smem,
                           cudaStream_t s, const NrLaunch *fb, size_t smem_optin) {
    ClRun a;
    a.dn = dn;
    a.dc = dc;
    a.m[0] = m0;
    a.m[1] = m1;
    a.fs0 = fs0;
    a.fs1 = fs1;
    a.tol = o.tol;
    a.max_iter = o.max_iter;
    a.flat = o.flat_start;
    a.vm = vm;
    a.va = va;
    a.ef = ef;
    a.iv = iv;
    a.bmax = bmax;
    a.res = res;
    a.fallback = 0;
    if (fb) {  // the Newton-Raphson fallback's layout, when it fits
        const size_t need = nr_args_within(*fb, smem, a.nr);
        if (need + 4096 <= smem_optin && (need == smem || fdpf_cl_fits(need))) {
            smem = need;
            a.fallback = 1;
        }
    }
    cudaError_t e = cudaFuncSetAttribute(k_fdpf_cl<kClCtas>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fdpf_cl<kClCtas>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClCtas);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_fdpf_cl<kClCtas>, a);
}

// Whether a cluster of kClCtas CTAs with `smem` bytes each can be resident.
bool fdpf_cl_fits(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k_fdpf_cl<kClCtas>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fdpf_cl<kClCtas>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClCtas);
    cfg.blockDim = dim3(kClThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, k_fdpf_cl<kClCtas>, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters >= 1;
}

}  // namespace gbpf
