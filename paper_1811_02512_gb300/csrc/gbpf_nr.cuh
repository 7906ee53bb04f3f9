// gbpf_nr.cuh -- the Newton-Raphson power flow of one case (Section III of
// arxiv 1811.02512) as device code shared by the Newton-Raphson kernels
// (gbpf_nr.cu) and the fast decoupled kernels, which fall back to it inside
// the same launch for cases the fast decoupled iteration leaves unconverged.
//
// Unknowns: (theta_i, V_i) of every non-slack bus i, one 2 x 2 block per
// entry of the bus-graph pattern of B' (the same ordering, elimination tree
// and levels).  The V unknown of a PV bus is pinned by an identity row and
// column, which keeps the block pattern equal to the bus graph.  The
// Jacobian is factorised without pivoting as J = L D U (unit block-lower L,
// unit block-upper U, 2 x 2 block diagonal D), column by column in level
// order with the same gather lists as the scalar LDL^T, and solved with the
// TMA-staged sweeps: J x = b uses L by rows and U by columns; J^T y = g uses
// U^T by rows and L^T by columns with the same factors (the adjoint).
#pragma once

#include "gbpf_device.cuh"

namespace gbpf {

// Arguments of the Newton-Raphson device code (by value in the kernels'
// parameters; the fast decoupled kernels carry one for their fallback).
struct NrArgs {
    DevNet dn;
    DevCases dc;
    DevMat m;          // pattern of B' (non-slack buses)
    void *F;           // [ncase][jstride] block factors (T)
    double *A;         // [ncase][jstride] FP64 Jacobian: D, Lc (J_rc), Uc (J_cr) regions
    int *fstat;        // [ncase] factor status of the last factorisation
    double tol;
    int max_iter;
    int flat;
    unsigned spin;
    int ir_max;
    double ir_tol, ir_abs;
    double *vm, *va;
    double *ef;        // [ncase][4 nbus]: e, f, P, Q
    double *xg;        // [ncase][6 nbus]: rhs (2n), refined x (2n), FP32 work (2n)
    double *bmax;      // [ncase][16]
    pf_case_result *res;
    const double *gva, *gvm;    // adjoint right-hand side per bus
    double *dJdP, *dJdQ;        // adjoint outputs per bus
    int use_smem;
    unsigned *jdone;   // [ncase][n] column done flags
    unsigned *jsync;   // [ncase][2] column counter, abort flag
    unsigned epoch0;   // factorisation k of this launch publishes epoch0 + k
    int fchunk;        // update terms staged per warp and pass (fits the shared memory)
};

// Fills `a` for launch L inside a kernel of 512 threads whose dynamic shared
// memory starts with the staging ring and holds `smem` bytes: the factor
// scratch after the ring takes as many staged update terms per warp as fit
// (32 to 128), the solve vector shares it when it fits.  Returns the
// reservation this needs: `smem`, or more when 32 terms do not fit.
size_t nr_args_within(const NrLaunch &L, size_t smem, NrArgs &a);

namespace {

constexpr int kNrChunkMax = 128;  // update terms staged per warp and pass in the block factor (at most)

// ------------------------------------------------------------ 2 x 2 blocks

template <class T>
struct B2 {
    T a, b, c, d;  // [[a, b], [c, d]]
};

template <class T>
__device__ __forceinline__ B2<T> ld2(const T *p) { return B2<T>{p[0], p[1], p[2], p[3]}; }

// A block written by another SM during this launch: read through L2.
template <class T>
__device__ __forceinline__ B2<T> ldcg2(const T *p) {
    return B2<T>{__ldcg(p), __ldcg(p + 1), __ldcg(p + 2), __ldcg(p + 3)};
}

template <class T>
__device__ __forceinline__ void st2(T *p, const B2<T> &m) {
    p[0] = m.a; p[1] = m.b; p[2] = m.c; p[3] = m.d;
}

template <class T>
__device__ __forceinline__ B2<T> mul2(const B2<T> &x, const B2<T> &y) {
    return B2<T>{x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c,
                 x.c * y.b + x.d * y.d};
}

// Injection terms of branch-aware admittance entry (i, k) of case `outage`:
// the base Y entry at Ybus position p minus the outaged branch's share.
__device__ __forceinline__ void y_entry(const DevNet &dn, int outage, int i, int k, int p,
                                        double &G, double &B) {
    G = p >= 0 ? dn.G[p] : 0.0;
    B = p >= 0 ? dn.B[p] : 0.0;
    if (outage < 0 || !dn.bstatus[outage]) return;
    const int f = dn.bf[outage], t = dn.bt[outage];
    if (!((i == f || i == t) && (k == f || k == t))) return;
    const double r = dn.br[outage], x = dn.bx[outage], bc = dn.bb[outage], tp = dn.btap[outage];
    const double den = r * r + x * x;
    const double ys_re = r / den, ys_im = -x / den;
    if (i != k) {
        G += ys_re / tp;
        B += ys_im / tp;
    } else if (i == f) {
        G -= ys_re / (tp * tp);
        B -= (ys_im + 0.5 * bc) / (tp * tp);
    } else {
        G -= ys_re;
        B -= ys_im + 0.5 * bc;
    }
}

// Off-diagonal Jacobian block J_ik = d(P_i, Q_i)/d(theta_k, V_k) from the
// rectangular voltages; PV rows/columns pinned.
__device__ __forceinline__ B2<double> jac_off(double G, double B, double ei, double fi, double ek,
                                              double fk, double vk, bool pv_i, bool pv_k) {
    const double a = ei * ek + fi * fk;  // V_i V_k cos(theta_ik)
    const double b = fi * ek - ei * fk;  // V_i V_k sin(theta_ik)
    B2<double> J;
    J.a = G * b - B * a;                 // dP_i / dtheta_k
    J.b = (G * a + B * b) / vk;          // dP_i / dV_k
    J.c = -(G * a + B * b);              // dQ_i / dtheta_k
    J.d = (G * b - B * a) / vk;          // dQ_i / dV_k
    if (pv_i) { J.c = 0.0; J.d = 0.0; }
    if (pv_k) { J.b = 0.0; J.d = 0.0; }
    return J;
}

__device__ __forceinline__ B2<double> jac_diag(double G, double B, double P, double Q, double v,
                                               bool pv) {
    B2<double> J;
    J.a = -Q - B * v * v;     // dP_i / dtheta_i
    J.b = P / v + G * v;      // dP_i / dV_i
    J.c = P - G * v * v;      // dQ_i / dtheta_i
    J.d = Q / v - B * v;      // dQ_i / dV_i
    if (pv) { J.b = 0.0; J.c = 0.0; J.d = 1.0; }
    return J;
}
// Rectangular voltages of the CTA's bus slice.
__device__ void nr_rect(const NrArgs &a, int c, int i0, int i1) {
    const int nbus = a.dn.nbus;
    const double *vm = a.vm + (long long)c * nbus;
    const double *va = a.va + (long long)c * nbus;
    double *e = a.ef + (long long)c * 4 * nbus;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        double s, co;
        sincos(va[i], &s, &co);
        e[i] = vm[i] * co;
        e[nbus + i] = vm[i] * s;
    }
}

// Injections, mismatch and Newton right-hand side of the slice; returns the
// CTA maximum (NaN wins).
__device__ double nr_mismatch_slice(const NrArgs &a, int c, int i0, int i1, double *red) {
    const DevNet &dn = a.dn;
    const int nbus = dn.nbus;
    const double *e = a.ef + (long long)c * 4 * nbus;
    const double *f = e + nbus;
    double *P = const_cast<double *>(e) + 2 * nbus;
    double *Q = P + nbus;
    double *rhs = a.xg + (long long)c * 6 * nbus;
    const int outage = a.dc.outage[c];
    double mx = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        double p, q;
        bus_injection(dn, i, outage, e, f, p, q);
        P[i] = p;
        Q[i] = q;
        const int t = dn.btype[i];
        const long long idx = (long long)c * nbus + i;
        const double dP = (t != PF_BUS_SLACK) ? a.dc.Psp[idx] - p : 0.0;
        const double dQ = (t == PF_BUS_PQ) ? a.dc.Qsp[idx] - q : 0.0;
        double l = fmax(fabs(dP), fabs(dQ));
        if (dP != dP || dQ != dQ) l = __longlong_as_double(0x7ff8000000000000ll);
        mx = nan_max(mx, l);
        const int k = a.m.new_of_bus[i];
        if (k >= 0) {
            rhs[2 * k] = dP;
            rhs[2 * k + 1] = dQ;
        }
    }
    return block_max(mx, red);
}

// FP64 Jacobian of case c into A: the diagonal blocks of the slots [s0, s1)
// of the (n + nnz) slot range and the lower / upper blocks of the others.
__device__ void nr_assemble(const NrArgs &a, int c, int s0, int s1) {
    const DevNet &dn = a.dn;
    const DevMat &m = a.m;
    const int nbus = dn.nbus;
    const double *e = a.ef + (long long)c * 4 * nbus;
    const double *f = e + nbus;
    const double *P = e + 2 * nbus;
    const double *Q = e + 3 * nbus;
    const double *vm = a.vm + (long long)c * nbus;
    double *A = a.A + (long long)c * m.jstride;
    const int outage = a.dc.outage[c];
    for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        if (s < m.n) {
            const int i = m.bus[s];
            double G, B;
            y_entry(dn, outage, i, i, dn.ydiag[i], G, B);
            st2(A + m.jD + 4 * s, jac_diag(G, B, P[i], Q[i], vm[i], dn.btype[i] == PF_BUS_PV));
        } else {
            const int p = s - m.n;
            int col = 0;
            {  // column of CSC slot p: binary search in Cp
                int lo = 0, hi = m.n;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (m.Cp[mid] <= p) lo = mid; else hi = mid;
                }
                col = lo;
            }
            const int r = m.Cr[p];
            const int i = m.bus[r], k = m.bus[col];
            const bool pvi = dn.btype[i] == PF_BUS_PV, pvk = dn.btype[k] == PF_BUS_PV;
            double G, B;
            y_entry(dn, outage, i, k, m.src[m.n + p], G, B);
            st2(A + m.jLc + 4 * p, jac_off(G, B, e[i], f[i], e[k], f[k], vm[k], pvi, pvk));
            y_entry(dn, outage, k, i, m.srcT[p], G, B);
            st2(A + m.jUc + 4 * p, jac_off(G, B, e[k], f[k], e[i], f[i], vm[i], pvk, pvi));
        }
    }
}

// Block LDU factor of the Jacobian of case c (Section III.B with 2 x 2
// blocks, no pivoting; the pivot check is on det(D_c) against the largest
// diagonal-block entry) by all C blocks of its cluster, driven by the
// elimination tree's dependencies: every warp of the cluster takes
// columns in level order from a counter, waits until the columns of row c of
// L are done (their flags hold `epoch`), then computes each target block of
// column c with a lane per target from the gather lists of the pattern
// (Section III.B, 2 x 2 blocks),
//   A_ic - sum_k L_ik (D_k U_kc),  A_ci - sum_k (L_ck D_k) U_ki,
// publishes D_c, D_c^-1, L_ic = A_ic D_c^-1, U_ci = D_c^-1 A_ci (by column
// and by row) and its own flag.  Every wait is bounded; one that gives up
// raises the case's abort flag.  Cluster-uniform status.
template <class T, int C>
__device__ int cluster_block_factor(const NrArgs &a, int c, int rank, T *F, const double *Aj,
                                    unsigned char *scratch, double *red, unsigned epoch) {
    const DevMat &m = a.m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int chunk = a.fchunk;
    const int sa = 8 * (m.max_col + 1) + 8 * chunk;
    T *accL = reinterpret_cast<T *>(scratch) + warp * sa;
    T *accU = accL + 4 * (m.max_col + 1);
    T *termL = accU + 4 * (m.max_col + 1);
    T *termU = termL + 4 * chunk;
    T *D = F + m.jD, *Di = F + m.jDi, *Lc = F + m.jLc, *Uc = F + m.jUc;
    T *Lr = F + m.jLr, *Ur = F + m.jUr;
    unsigned *done = a.jdone + (long long)c * m.n;
    unsigned *ctr = a.jsync + 2LL * c, *abort_flag = ctr + 1;
    // pivot tolerance: largest diagonal-block entry over the cluster
    const int nd = 4 * m.n, slice = (nd + C - 1) / C;
    double amax = 0.0;
    for (int j = rank * slice + int(threadIdx.x); j < min(nd, (rank + 1) * slice); j += blockDim.x)
        amax = fmax(amax, fabs(Aj[m.jD + j]));
    amax = block_max(amax, red);
    if (threadIdx.x == 0) {
        a.bmax[(long long)c * 16 + rank] = amax;
        if (rank == 0) {
            *ctr = 0u;
            *abort_flag = 0u;
            a.fstat[c] = PF_OK;
        }
    }
    cluster_sync<C>();
    amax = 0.0;
    for (int r = 0; r < C; r++) amax = fmax(amax, a.bmax[(long long)c * 16 + r]);
    const double piv = 1e-14 * amax * amax;
    for (;;) {
        unsigned col = 0;
        if (lane == 0) col = atomicAdd(ctr, 1u);
        col = __shfl_sync(0xffffffffu, col, 0);
        if (col >= unsigned(m.n)) break;
        const int cc = int(col);
        bool ok = true;
        for (int q = m.Fp[cc] + lane; q < m.Fp[cc + 1] && ok; q += 32) {
            const unsigned *f = done + m.Fc[q];
            unsigned it = 0;
            unsigned v;
            for (;;) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
                if (v == epoch) break;
                if (++it > a.spin || *reinterpret_cast<volatile unsigned *>(abort_flag)) {
                    ok = false;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) {
                atomicExch(abort_flag, 1u);
                atomicCAS(a.fstat + c, PF_OK, PF_ERR_TIMEOUT);
            }
            continue;
        }
        const int c0 = m.Cp[cc], cnt = m.Cp[cc + 1] - c0, tb = c0 + cc;
        for (int t = lane; t <= cnt; t += 32) {
            const double *src = t == 0 ? Aj + m.jD + 4 * cc : Aj + m.jLc + 4 * (c0 + t - 1);
            st2(accL + 4 * t, B2<T>{T(src[0]), T(src[1]), T(src[2]), T(src[3])});
            if (t > 0) {
                const double *us = Aj + m.jUc + 4 * (c0 + t - 1);
                st2(accU + 4 * t, B2<T>{T(us[0]), T(us[1]), T(us[2]), T(us[3])});
            }
        }
        // the column's update terms, a chunk at a time: evaluated with the
        // whole warp (a lane per term) into shared memory, then summed per
        // target with a lane per target in list order
        const int gb = m.gp[tb], ge = m.gp[tb + cnt + 1];
        for (int cb = gb; cb < ge; cb += chunk) {
            const int ce = min(ge, cb + chunk);
            // four terms per lane in flight: their indices, then their blocks
            for (int g0 = cb + lane; g0 < ce; g0 += 128) {
                int4 e[4];
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (g0 + 32 * u < ce) e[u] = __ldg(m.gl + g0 + 32 * u);
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int g = g0 + 32 * u;
                    if (g >= ce) continue;
                    const B2<T> Lx = ldcg2(Lc + 4 * e[u].x), Dk = ldcg2(D + 4 * e[u].z);
                    const B2<T> Uy = ldcg2(Uc + 4 * e[u].y), Ly = ldcg2(Lc + 4 * e[u].y);
                    const B2<T> Ux = ldcg2(Uc + 4 * e[u].x);
                    st2(termL + 4 * (g - cb), mul2(Lx, mul2(Dk, Uy)));
                    st2(termU + 4 * (g - cb), mul2(mul2(Ly, Dk), Ux));
                }
            }
            __syncwarp();
            for (int t = lane; t <= cnt; t += 32) {
                const int lo = max(m.gp[tb + t], cb), hi = min(m.gp[tb + t + 1], ce);
                if (lo >= hi) continue;
                B2<T> sl{T(0), T(0), T(0), T(0)}, su{T(0), T(0), T(0), T(0)};
                for (int g = lo; g < hi; g++) {
                    const B2<T> a2 = ld2(termL + 4 * (g - cb)), b2 = ld2(termU + 4 * (g - cb));
                    sl.a += a2.a; sl.b += a2.b; sl.c += a2.c; sl.d += a2.d;
                    su.a += b2.a; su.b += b2.b; su.c += b2.c; su.d += b2.d;
                }
                T *al = accL + 4 * t;
                al[0] -= sl.a; al[1] -= sl.b; al[2] -= sl.c; al[3] -= sl.d;
                if (t > 0) {
                    T *au = accU + 4 * t;
                    au[0] -= su.a; au[1] -= su.b; au[2] -= su.c; au[3] -= su.d;
                }
            }
            __syncwarp();
        }
        const B2<T> Dc = ld2(accL);
        const T det = Dc.a * Dc.d - Dc.b * Dc.c;
        const B2<T> inv{Dc.d / det, -Dc.b / det, -Dc.c / det, Dc.a / det};
        if (lane == 0) {
            st2(D + 4 * cc, Dc);
            st2(Di + 4 * cc, inv);
            const double dd = double(det);
            if (!isfinite(dd) || !isfinite(double(Dc.a)) || !isfinite(double(Dc.d)))
                atomicCAS(a.fstat + c, PF_OK, PF_ERR_NONFINITE);
            else if (fabs(dd) <= piv)
                atomicCAS(a.fstat + c, PF_OK, PF_ERR_SINGULAR);
        }
        for (int t = lane; t < cnt; t += 32) {
            const B2<T> L = mul2(ld2(accL + 4 * (1 + t)), inv);
            const B2<T> U = mul2(inv, ld2(accU + 4 * (1 + t)));
            st2(Lc + 4 * (c0 + t), L);
            st2(Uc + 4 * (c0 + t), U);
            const int q = m.Cpos[c0 + t];
            st2(Lr + 4 * q, L);
            st2(Ur + 4 * q, U);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(done + cc), "r"(epoch) : "memory");
    }
    cluster_sync<C>();
    const int st = *reinterpret_cast<volatile int *>(a.fstat + c);
    cluster_sync<C>();
    return st;
}

// J x = x (TRANS = false) or J^T x = x (TRANS = true) with the block factors.
template <class T, class X, bool TRANS>
__device__ bool block_solve2(Ring *R, unsigned char *stages, const DevMat &m, const T *F, X *x,
                             unsigned spin) {
    if (!staged_sweep<T, X, 2, TRANS>(R, stages, m.pfJ, m.npfJ, m.Fp, m.Fc,
                                      F + (TRANS ? m.jUr : m.jLr), nullptr, m.lvl_ptr, x, spin))
        return false;
    return staged_sweep<T, X, 2, TRANS>(R, stages, m.pbJ, m.npbJ, m.Cp, m.Cr,
                                        F + (TRANS ? m.jLc : m.jUc), F + m.jDi, m.lvl_ptr, x, spin);
}

// r = b - J x (TRANS: b - J^T x) for row r of the FP64 Jacobian A.
template <bool TRANS>
__device__ __forceinline__ void jac_residual_row(const DevMat &m, const double *A, const double *b,
                                                 const double *x, int r, double &r0, double &r1) {
    double s0 = b[2 * r], s1 = b[2 * r + 1];
    const double *D = A + m.jD + 4 * r;
    const double x0 = x[2 * r], x1 = x[2 * r + 1];
    if (!TRANS) {
        s0 -= D[0] * x0 + D[1] * x1;
        s1 -= D[2] * x0 + D[3] * x1;
    } else {
        s0 -= D[0] * x0 + D[2] * x1;
        s1 -= D[1] * x0 + D[3] * x1;
    }
    // entries of row r with columns c < r (CSR), and i > r (CSC of column r)
    for (int q = m.Fp[r]; q < m.Fp[r + 1]; q++) {
        const int c = m.Fc[q], p = m.Fpos[q];
        const double *Bk = A + (TRANS ? m.jUc : m.jLc) + 4 * p;  // J_rc, or J_cr for J^T
        const double y0 = x[2 * c], y1 = x[2 * c + 1];
        if (!TRANS) { s0 -= Bk[0] * y0 + Bk[1] * y1; s1 -= Bk[2] * y0 + Bk[3] * y1; }
        else { s0 -= Bk[0] * y0 + Bk[2] * y1; s1 -= Bk[1] * y0 + Bk[3] * y1; }
    }
    for (int p = m.Cp[r]; p < m.Cp[r + 1]; p++) {
        const int i = m.Cr[p];
        const double *Bk = A + (TRANS ? m.jLc : m.jUc) + 4 * p;  // J_ri, or J_ir for J^T
        const double y0 = x[2 * i], y1 = x[2 * i + 1];
        if (!TRANS) { s0 -= Bk[0] * y0 + Bk[1] * y1; s1 -= Bk[2] * y0 + Bk[3] * y1; }
        else { s0 -= Bk[0] * y0 + Bk[2] * y1; s1 -= Bk[1] * y0 + Bk[3] * y1; }
    }
    r0 = s0;
    r1 = s1;
}

// Refined block solve of case c in one block: x = J^-1 b (or J^-T b) into
// the refined-x region, with FP64 residuals against A when the factor is
// FP32 (or when `always_refine`, e.g. factors of an earlier state).
template <class T, bool TRANS>
__device__ bool nr_solve(const NrArgs &a, Ring *R, unsigned char *stages, T *xs, const T *F,
                         const double *A, int c, double *red, int &ir_steps, bool always_refine) {
    const DevMat &m = a.m;
    const int nbus = a.dn.nbus;
    const int N = 2 * m.n;
    double *b = a.xg + (long long)c * 6 * nbus;
    double *x64 = b + 2 * nbus;
    T *xv = xs ? xs : reinterpret_cast<T *>(x64 + 2 * nbus);
    const bool refine = always_refine || sizeof(T) != sizeof(double);
    double bn = 0.0;
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
        xv[r] = T(b[r]);
        bn = fmax(bn, fabs(b[r]));
    }
    bn = block_max(bn, red);
    bool ok = true;
    for (int k = 0;; k++) {
        ok = block_solve2<T, T, TRANS>(R, stages, m, F, xv, a.spin);
        if (!ok) break;
        for (int r = threadIdx.x; r < N; r += blockDim.x)
            x64[r] = (k == 0 ? 0.0 : x64[r]) + double(xv[r]);
        __syncthreads();
        if (!refine || k >= a.ir_max) break;
        double rn = 0.0;
        for (int r = threadIdx.x; r < m.n; r += blockDim.x) {
            double r0, r1;
            jac_residual_row<TRANS>(m, A, b, x64, r, r0, r1);
            xv[2 * r] = T(r0);
            xv[2 * r + 1] = T(r1);
            rn = nan_max(rn, fmax(fabs(r0), fabs(r1)));
        }
        rn = block_max(rn, red);
        if (!(rn > a.ir_tol * bn) || !(rn > a.ir_abs)) break;
        ir_steps++;
    }
    return ok;
}

// Newton-Raphson power flow of one case per cluster of C CTAs: mismatch,

// Newton-Raphson power flow of case c on the C CTAs of its cluster (this
// CTA is `rank`): mismatch, Jacobian assembly and factor spread over the
// cluster, the refined solve in CTA 0, until the mismatch is within a.tol or
// a.max_iter steps; writes the case's result (method PF_NR).  Shared memory:
// the staging ring at smem_raw, then the factor scratch (a.fchunk update
// terms per warp), which the solve vector shares when a.use_smem.  The ring
// R must be initialised; its phases run on from whatever used it before.
template <class T, int C>
__device__ __forceinline__ void nr_case(const NrArgs &a, int c, int rank, unsigned char *smem_raw,
                                        double *red, Ring *R) {
    const DevNet &dn = a.dn;
    const DevMat &m = a.m;
    const int nbus = dn.nbus;
    unsigned char *stages = smem_raw;
    unsigned char *scratch = smem_raw + kStages * kStageBytes;
    T *xs = a.use_smem ? reinterpret_cast<T *>(scratch) : nullptr;  // shares the factor scratch
    double *vm = a.vm + (long long)c * nbus;
    double *va = a.va + (long long)c * nbus;
    double *flag = a.bmax + (long long)c * 16 + 15;
    T *F = static_cast<T *>(a.F) + (long long)c * m.jstride;
    const double *A = a.A + (long long)c * m.jstride;
    const int slice = (nbus + C - 1) / C;
    const int i0 = rank * slice, i1 = min(nbus, i0 + slice);
    const int nslot = m.n + m.nnz;
    const int sslice = (nslot + C - 1) / C;
    const int s0 = rank * sslice, s1 = min(nslot, s0 + sslice);
    if (a.flat)
        for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const int t = dn.btype[i];
            vm[i] = (t == PF_BUS_PQ) ? 1.0 : dn.vset[i];
            va[i] = (t == PF_BUS_SLACK) ? dn.va0[i] : 0.0;
        }
    int status = PF_ERR_NOT_CONVERGED, iters = 0, ir_steps = 0;
    double mis = INFINITY;
    for (int it = 0;; it++) {
        nr_rect(a, c, i0, i1);
        cluster_sync<C>();
        const double mx = nr_mismatch_slice(a, c, i0, i1, red);
        if (threadIdx.x == 0) a.bmax[(long long)c * 16 + rank] = mx;
        cluster_sync<C>();
        mis = 0.0;
        for (int r = 0; r < C; r++) mis = nan_max(mis, a.bmax[(long long)c * 16 + r]);
        if (!isfinite(mis)) { status = PF_ERR_NONFINITE; break; }
        if (mis <= a.tol) { status = PF_OK; break; }
        if (it >= a.max_iter) break;
        nr_assemble(a, c, s0, s1);
        cluster_sync<C>();
        const int fs = cluster_block_factor<T, C>(a, c, rank, F, A, scratch, red, a.epoch0 + unsigned(it) + 1u);
        if (rank == 0) {
            bool ok = fs == PF_OK;
            if (ok) ok = nr_solve<T, false>(a, R, stages, xs, F, A, c, red, ir_steps, false);
            if (threadIdx.x == 0) {
                a.fstat[c] = fs;
                *flag = fs != PF_OK ? double(fs) : (ok ? 0.0 : double(PF_ERR_TIMEOUT));
            }
        }
        cluster_sync<C>();
        if (*flag != 0.0) { status = int(*flag); break; }
        const double *dx = a.xg + (long long)c * 6 * nbus + 2 * nbus;
        for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const int k = m.new_of_bus[i];
            if (k >= 0) {
                va[i] += dx[2 * k];
                if (dn.btype[i] == PF_BUS_PQ) vm[i] += dx[2 * k + 1];
            }
        }
        iters++;
    }
    if (rank == 0 && threadIdx.x == 0) {
        a.res[c].status = status;
        a.res[c].iters = iters;
        a.res[c].ir_steps = ir_steps;
        a.res[c].method = PF_NR;
        a.res[c].max_mismatch = mis;
    }
    cluster_sync<C>();
}

// The Newton-Raphson fallback of case c inside a fast decoupled kernel, out
// of line: the fast decoupled loop keeps its own register allocation, and
// the arguments are read where they are (a __grid_constant__ parameter or a
// global array).  The caller's status is cluster-uniform, so every CTA of
// the cluster enters.
template <class T, int C>
__device__ __noinline__ void nr_fallback(const NrArgs &a, int c, int rank, unsigned char *smem_raw,
                                         double *red, Ring *R) {
    nr_case<T, C>(a, c, rank, smem_raw, red, R);
}

}  // namespace

}  // namespace gbpf
