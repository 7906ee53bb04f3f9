// gbpf_batch.cu -- lockstep batched fast-decoupled power flow ("lane engine").
//
// A batch of cases of one topology shares the symbolic factorisation: the
// same elimination tree, the same levels, the same index arrays.  Here 32
// cases form a lane group and advance together: every level of a
// substitution (Section III.C of arxiv 1811.02512) is walked once for the 32
// cases of a group, one case per lane, so the level-to-level latency of the
// hierarchical schedule (Section II.B) is paid once per 32 cases.  Load
// scenarios share one factor (values broadcast to the lanes); branch-outage
// cases carry their own factor, stored lane-interleaved [slot][32] so the
// lanes of a warp read one 128-byte line per entry.  The FP64 nodal mismatch
// (Section II.A) runs over all (bus, case) pairs of the batch with the state
// laid out [bus][case], so the admittance values are broadcast and the
// voltages read coalesced.  One P/Q half-iteration pair is a short sequence
// of kernels that the host captures once in a CUDA graph and replays until
// every case has converged.
#include "gbpf_device.cuh"

namespace gbpf {

namespace {

constexpr int kLanes = 32;
constexpr int kLaneThreads = 512;

struct LaneArgs {
    DevNet dn;
    DevCases dc;
    DevMat m0, m1;
    LaneSet L;
    const void *F0, *F1;   // per-instance factors (instance 0 serves the shared groups)
    const int *fs0, *fs1;  // per-instance factor status
    const double *A0, *A1; // per-instance FP64 values (refinement residuals)
    double tol;
    int flat;
    unsigned spin;
};

__device__ __forceinline__ const DevMat &mat(const LaneArgs &a, int which) { return which ? a.m1 : a.m0; }

// ------------------------------------------------------------ layout moves

// Start of a batch run: lane state from the case-major inputs, flat start,
// trigonometry, 1/V, rectangular voltages; lanes whose factors failed are
// retired with the factor status.
__global__ void k_lane_load(LaneArgs a, const double *vm, const double *va) {
    const LaneSet &L = a.L;
    const int nbus = a.dn.nbus;
    const long long total = (long long)nbus * L.ncp;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = int(idx / L.ncp), lane = int(idx % L.ncp);
        const int c = L.gcase[lane];
        double v = 1.0, t = 0.0, ps = 0.0, qs = 0.0;
        if (c >= 0) {
            const int bt = a.dn.btype[i];
            if (a.flat) {
                v = bt == PF_BUS_PQ ? 1.0 : a.dn.vset[i];
                t = bt == PF_BUS_SLACK ? a.dn.va0[i] : 0.0;
            } else {
                v = vm[(long long)c * nbus + i];
                t = va[(long long)c * nbus + i];
            }
            ps = a.dc.Psp[(long long)c * nbus + i];
            qs = a.dc.Qsp[(long long)c * nbus + i];
        }
        double s, co;
        sincos(t, &s, &co);
        L.vm[idx] = v;
        L.va[idx] = t;
        L.cs[idx] = co;
        L.sn[idx] = s;
        L.iv[idx] = 1.0 / v;
        L.e[idx] = v * co;
        L.f[idx] = v * s;
        L.psp[idx] = ps;
        L.qsp[idx] = qs;
        if (i == 0) {
            int st = c >= 0 ? PF_ERR_NOT_CONVERGED : PF_OK;
            if (c >= 0) {
                const int inst = a.dc.inst[c];
                if (a.fs0[inst] != PF_OK) st = a.fs0[inst];
                else if (a.fs1[inst] != PF_OK) st = a.fs1[inst];
            }
            L.status[lane] = st;
            L.active[lane] = st == PF_ERR_NOT_CONVERGED ? 1 : 0;
            L.iters[lane] = 0;
            L.irs[lane] = 0;
            L.maxmis[lane] = 0.0;
            L.lastmis[lane] = INFINITY;
        }
    }
}

// End of a batch run: case-major state and per-case results.
__global__ void k_lane_store(LaneArgs a, double *vm, double *va, pf_case_result *res) {
    const LaneSet &L = a.L;
    const int nbus = a.dn.nbus;
    const long long total = (long long)nbus * L.ncp;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = int(idx / L.ncp), lane = int(idx % L.ncp);
        const int c = L.gcase[lane];
        if (c < 0) continue;
        vm[(long long)c * nbus + i] = L.vm[idx];
        va[(long long)c * nbus + i] = L.va[idx];
        if (i == 0) {
            res[c].status = L.status[lane];
            res[c].iters = L.iters[lane];
            res[c].ir_steps = L.irs[lane];
            res[c].method = PF_FDPF;
            res[c].max_mismatch = L.lastmis[lane];
        }
    }
}

// Own-factor groups: the per-instance factors of their lanes, interleaved
// [slot][32] (empty lanes copy instance 0).
template <class T>
__global__ void k_lane_factors(LaneArgs a, int which, T *LF) {
    const DevMat &m = mat(a, which);
    const T *F = static_cast<const T *>(which ? a.F1 : a.F0);
    const LaneSet &L = a.L;
    const long long per = (long long)m.stride * kLanes;
    const long long total = per * L.nown;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int go = int(idx / per);
        const long long rem = idx % per;
        const int s = int(rem / kLanes), l = int(rem % kLanes);
        const int g = L.owngroup[go];
        const int inst = L.ginst[g * kLanes + l];
        LF[idx] = F[(long long)inst * m.stride + s];
    }
}

// ------------------------------------------------------------ Section II.A

// Mismatch of one half-iteration for every active (bus, case): one warp per
// bus and group, one lane per case; dP/V or dQ/V is written to the group's
// right-hand side (FP64 and the solve precision) in level order; the
// per-case maximum goes to maxmis through an atomic maximum.
template <class T>
__global__ void __launch_bounds__(256) k_lane_mismatch(LaneArgs a, int which) {
    __shared__ double red[8][kLanes];
    const LaneSet &L = a.L;
    const DevNet &dn = a.dn;
    const int nbus = dn.nbus;
    const int g = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + warp;
    const int idxl = g * kLanes + lane;
    const int c = L.gcase[idxl];
    double mx = 0.0;
    if (i < nbus && c >= 0 && L.active[idxl]) {
        const long long ncp = L.ncp;
        double ir = 0.0, ii = 0.0;
        for (int p = dn.rowptr[i]; p < dn.rowptr[i + 1]; p++) {
            const long long k = (long long)dn.col[p] * ncp + idxl;
            const double gg = dn.G[p], bb = dn.B[p];
            const double ek = L.e[k], fk = L.f[k];
            ir += gg * ek - bb * fk;
            ii += gg * fk + bb * ek;
        }
        const long long ki = (long long)i * ncp + idxl;
        const double ei = L.e[ki], fi = L.f[ki];
        const int outage = a.dc.outage[c];
        if (outage >= 0 && dn.bstatus[outage] && (i == dn.bf[outage] || i == dn.bt[outage])) {
            const double r = dn.br[outage], x = dn.bx[outage], bc = dn.bb[outage], t = dn.btap[outage];
            const double den = r * r + x * x;
            const double ys_re = r / den, ys_im = -x / den;
            const int o = (i == dn.bf[outage]) ? dn.bt[outage] : dn.bf[outage];
            const long long ko = (long long)o * ncp + idxl;
            double gs, bs;
            if (i == dn.bf[outage]) {
                gs = ys_re / (t * t);
                bs = (ys_im + 0.5 * bc) / (t * t);
            } else {
                gs = ys_re;
                bs = ys_im + 0.5 * bc;
            }
            const double gm = -ys_re / t, bm = -ys_im / t;
            ir -= gs * ei - bs * fi + gm * L.e[ko] - bm * L.f[ko];
            ii -= gs * fi + bs * ei + gm * L.f[ko] + bm * L.e[ko];
        }
        const double P = ei * ir + fi * ii;
        const double Q = fi * ir - ei * ii;
        const int bt = dn.btype[i];
        const double dP = bt != PF_BUS_SLACK ? L.psp[ki] - P : 0.0;
        const double dQ = bt == PF_BUS_PQ ? L.qsp[ki] - Q : 0.0;
        mx = fmax(fabs(dP), fabs(dQ));
        if (dP != dP || dQ != dQ) mx = __longlong_as_double(0x7ff8000000000000ll);
        const int k = mat(a, which).new_of_bus[i];
        if (k >= 0) {
            const double rhs = (which == 0 ? dP : dQ) * L.iv[ki];
            const long long q = ((long long)g * nbus + k) * kLanes + lane;
            L.b[q] = rhs;
            static_cast<T *>(L.X)[q] = T(rhs);
        }
    }
    red[warp][lane] = mx;
    __syncthreads();
    if (warp == 0) {
        double m = red[0][lane];
        for (int w = 1; w < 8; w++) m = nan_max(m, red[w][lane]);
        if (c >= 0 && m != 0.0) atomic_max_nonneg(&L.maxmis[idxl], m);
    }
}

// Convergence of every case from its maximum (checked before each half-step):
// finished lanes retire; the maximum is reset and the still-active lanes are
// counted for the host.
__global__ void k_lane_check(LaneArgs a) {
    const LaneSet &L = a.L;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L.ncp) return;
    if (L.gcase[idx] < 0 || !L.active[idx]) return;
    const double m = L.maxmis[idx];
    L.maxmis[idx] = 0.0;
    L.lastmis[idx] = m;
    if (!isfinite(m)) {
        L.status[idx] = PF_ERR_NONFINITE;
        L.active[idx] = 0;
    } else if (m <= a.tol) {
        L.status[idx] = PF_OK;
        L.active[idx] = 0;
    } else {
        atomicAdd(L.nactive, 1);
    }
}

// ------------------------------------------------------------ Section III.C

// Rows of one staged piece for the W cases of a solve group, whose vectors
// x[row][W] live in shared memory.  Values (and, in the back substitution,
// the inverse diagonal) come from the stage (shared factor) or from the
// interleaved own factors lf[(slot) * 32 + lane] (lanes of the group).
// mode 0/1: thread per (row, case); mode 2: warp 0 alone walks the narrow
// levels of the piece, in groups of lanes per (row, case) with the entries
// split over the group and summed by shuffles; mode 3: part of one row.
template <class T, int W>
__device__ __forceinline__ void lane_piece(const int *h, const unsigned char *base, T *x,
                                           const T *lfv, const T *lfd, int mode) {
    const int *P = reinterpret_cast<const int *>(base);
    const int *I = reinterpret_cast<const int *>(base + h[6]);
    const T *Vs = reinterpret_cast<const T *>(base + h[7]);
    const T *Ds = h[10] >= 0 ? reinterpret_cast<const T *>(base + h[10]) : nullptr;
    const int r0 = h[0], r1 = h[1], p_lo = h[3], i_lo = h[4], v_lo = h[5], d_lo = h[11];
    const bool back = Ds != nullptr || lfd != nullptr;
    auto val = [&](int e, int l) -> T { return lfv ? lfv[(long long)e * kLanes + l] : Vs[e - v_lo]; };
    auto dinv = [&](int r, int l) -> T { return lfd ? lfd[(long long)r * kLanes + l] : Ds[r - d_lo]; };
    if (mode <= 1) {
        const int npair = (r1 - r0) * W;
        for (int t = threadIdx.x; t < npair; t += blockDim.x) {
            const int r = r0 + t / W, l = t % W;
            T s = x[r * W + l];
            if (back) s *= dinv(r, l);
            for (int e = P[r - p_lo]; e < P[r + 1 - p_lo]; e++) s -= val(e, l) * x[I[e - i_lo] * W + l];
            x[r * W + l] = s;
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    auto rows_grouped = [&](int ra, int rb, int ea, int eb, bool first) {
        const int npair = (rb - ra) * W;
        const int gsz = npair <= 1 ? 32 : npair <= 2 ? 16 : npair <= 4 ? 8 : npair <= 8 ? 4 : npair <= 16 ? 2 : 1;
        const int per = 32 / gsz;
        for (int p0 = 0; p0 < npair; p0 += per) {
            const int pr = p0 + lane / gsz, gl = lane % gsz;
            T acc = T(0);
            int r = -1, l = 0;
            if (pr < npair) {
                r = ra + pr / W;
                l = pr % W;
                const int a = ea >= 0 ? ea : P[r - p_lo], b = eb >= 0 ? eb : P[r + 1 - p_lo];
                for (int e = a + gl; e < b; e += gsz) acc += val(e, l) * x[I[e - i_lo] * W + l];
            }
            for (int o = gsz >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (r >= 0 && gl == 0) {
                T s = x[r * W + l];
                if (back && first) s *= dinv(r, l);
                x[r * W + l] = s - acc;
            }
        }
    };
    if (mode == 3) {
        rows_grouped(r0, r0 + 1, h[2], h[16], h[2] == P[r0 - p_lo]);
        return;
    }
    const int *LP = reinterpret_cast<const int *>(base + h[12]) - h[13];
    const int l0 = h[14], l1 = h[15];
    for (int li = 0; li <= l1 - l0; li++) {
        const int lv = back ? l1 - li : l0 + li;
        rows_grouped(max(LP[lv], r0), min(LP[lv + 1], r1), -1, -1, true);
        __syncwarp();
    }
}

// One substitution sweep for a solve group.  Thread 0 issues the copies:
// the first kStages pieces up front, then piece j + kStages once piece j
// has been consumed.  Block-wide pieces end with a block barrier that
// releases their stage; runs of single-warp pieces are consumed by warp 0,
// which issues the refills as it goes, while the other warps wait for the
// piece after the run.  Giving up is collective, as in staged_sweep: every
// thread waits (bounded) for the next piece and peeks at its control words,
// then one __syncthreads_or decides for all whether anyone's wait gave up;
// a header is acted on only after that vote, and a run ends with a vote of
// its own before the next piece is waited for.  After the sweep, if anything
// gave up, thread 0 waits for every copy that may still be in flight.
template <class T, int W>
__device__ bool lane_sweep(Ring *R, unsigned char *stages, const Piece *pieces, int np,
                           const int *ptr, const int *idx, const T *val, const T *dinv,
                           const int *lvl_ptr, T *x, const T *lfv, const T *lfd, unsigned spin) {
    const unsigned g0 = R->gcount;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *err = &R->err;
    int issued = 0;
    Piece next{};
    if (threadIdx.x == 0) {
        const int pre = np < kStages ? np : kStages;
        for (int j = 0; j < pre; j++)
            ring_issue<T, 1>(R, stages, int((g0 + j) % kStages), pieces[j], ptr, idx, val, dinv, lvl_ptr);
        issued = pre;
        if (kStages < np) next = pieces[kStages];
    }
    auto issue_after = [&](int j) {
        if (j + kStages < np) {
            ring_issue<T, 1>(R, stages, int((g0 + j) % kStages), next, ptr, idx, val, dinv, lvl_ptr);
            issued = j + kStages + 1;
            if (j + kStages + 1 < np) next = pieces[j + kStages + 1];
        }
    };
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
    bool stop = np > 0 ? __syncthreads_or(!wait_peek(0, mode, run_end) || *err != 0) != 0 : false;
    int j = 0;
    while (!stop && j < np) {
        const int st = int((g0 + unsigned(j)) % kStages);
        const bool run = mode >= 2;
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
                    lane_piece<T, W>(R->hdr[s2], stages + size_t(s2) * kStageBytes, x, lfv, lfd,
                                     R->hdr[s2][8]);
                    __syncwarp();
                    if (lane == 0) issue_after(jj);
                }
                if (fail && lane == 0) atomicExch(&R->err, 1);
            }
            // the others wait for warp 0 before waiting for the piece after
            // the run (its stage's previous phase must be complete first)
            if (__syncthreads_or(fail || *err != 0)) {
                stop = true;
                break;
            }
        } else {
            lane_piece<T, W>(R->hdr[st], stages + size_t(st) * kStageBytes, x, lfv, lfd, mode);
        }
        int nmode = 0, nrun = 0;
        const bool got = jn < np ? wait_peek(jn, nmode, nrun) : true;
        stop = __syncthreads_or(!got || *err != 0) != 0;
        if (!run && !stop && threadIdx.x == 0) issue_after(j);
        mode = nmode;
        run_end = nrun;
        j = jn;
    }
    if (stop && threadIdx.x == 0) atomicExch(&R->err, 1);
    __syncthreads();
    const bool ok = R->err == 0;
    if (!ok && threadIdx.x == 0) {
        // the caller's limit may be short; the drain always waits long
        // enough for a copy to land (a copy must not outlive the block)
        for (int q = (issued > kStages ? issued - kStages : 0); q < issued; q++) {
            const unsigned gq = g0 + unsigned(q);
            mbar_wait_bounded(&R->bar[gq % kStages], (gq / kStages) & 1u, spin > kDefaultSpin ? spin : kDefaultSpin);
        }
    }
    if (threadIdx.x == 0) R->gcount = g0 + unsigned(np);
    __syncthreads();
    return ok;
}

// L D L^T x = x for the W cases of solve group blockIdx.x (lanes
// [W blockIdx.x, W blockIdx.x + W) of the batch): the right-hand sides are
// staged into shared memory, solved, and x64 = (accumulate ? x64 : 0) + x.
template <class T, int W>
__global__ void __launch_bounds__(kLaneThreads) k_lane_solve(LaneArgs a, int which, int accumulate) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Ring R;
    const LaneSet &L = a.L;
    const DevMat &m = mat(a, which);
    const int nbus = a.dn.nbus;
    const int lane0 = blockIdx.x * W;
    const int g = lane0 / kLanes, lo = lane0 % kLanes;
    const bool shared = L.gshared[g] != 0;
    const T *F = static_cast<const T *>(which ? a.F1 : a.F0);  // instance 0
    const T *LF = shared ? nullptr
                         : static_cast<const T *>(which ? L.LF1 : L.LF0) +
                               (long long)L.gown[g] * m.stride * kLanes + lo;
    T *Xg = static_cast<T *>(L.X) + (long long)g * nbus * kLanes + lo;
    T *x = reinterpret_cast<T *>(smem_raw + kStages * kStageBytes);
    ring_init(&R);
    for (int t = threadIdx.x; t < m.n * W; t += blockDim.x) x[t] = Xg[(long long)(t / W) * kLanes + t % W];
    __syncthreads();
    bool ok = lane_sweep<T, W>(&R, smem_raw, m.pf, m.npf, m.Fp, m.Fc, shared ? F + m.offLr : nullptr,
                               nullptr, m.lvl_ptr, x,
                               shared ? nullptr : LF + (long long)m.offLr * kLanes, nullptr, a.spin);
    if (ok)
        ok = lane_sweep<T, W>(&R, smem_raw, m.pb, m.npb, m.Cp, m.Cr, shared ? F + m.offLc : nullptr,
                              shared ? F + m.offDi : nullptr, m.lvl_ptr, x,
                              shared ? nullptr : LF + (long long)m.offLc * kLanes,
                              shared ? nullptr : LF + (long long)m.offDi * kLanes, a.spin);
    double *x64 = L.x64 + (long long)g * nbus * kLanes + lo;
    for (int t = threadIdx.x; t < m.n * W; t += blockDim.x) {
        const long long q = (long long)(t / W) * kLanes + t % W;
        Xg[q] = x[t];
        x64[q] = (accumulate ? x64[q] : 0.0) + double(x[t]);
    }
    if (!ok && threadIdx.x < W) {
        const int idxl = lane0 + threadIdx.x;
        if (L.gcase[idxl] >= 0 && L.active[idxl]) {
            L.status[idxl] = PF_ERR_TIMEOUT;
            L.active[idxl] = 0;
        }
    }
}

// FP64 residual of the last solve, r = b - A x64 (A the FP64 values of each
// lane's instance), stored in the solve precision as the next right-hand side.
template <class T>
__global__ void __launch_bounds__(256) k_lane_resid(LaneArgs a, int which) {
    const LaneSet &L = a.L;
    const DevMat &m = mat(a, which);
    const int nbus = a.dn.nbus;
    const int g = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * 8 + warp;
    if (r >= m.n) return;
    const int idxl = g * kLanes + lane;
    const int inst = L.ginst[idxl];
    const double *A = (which ? a.A1 : a.A0) + (long long)inst * m.stride;
    const long long base = (long long)g * nbus * kLanes;
    const long long q = base + (long long)r * kLanes + lane;
    double s = L.b[q] - A[r] * L.x64[q];
    for (int e = m.Ap[r]; e < m.Ap[r + 1]; e++)
        s -= A[m.Apos[e]] * L.x64[base + (long long)m.Aj[e] * kLanes + lane];
    static_cast<T *>(L.X)[q] = T(s);
}

// State update of one half-iteration for every active (bus, case):
// theta += dtheta (cached cos/sin rotated by the small step, re-evaluated
// exactly near convergence or for large steps) or V += dV (1/V refreshed),
// then the rectangular voltages.
__global__ void k_lane_update(LaneArgs a, int which, int nir) {
    const LaneSet &L = a.L;
    const int nbus = a.dn.nbus;
    const long long total = (long long)nbus * L.ncp;
    const DevMat &m = mat(a, which);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = int(idx / L.ncp), lane = int(idx % L.ncp);
        if (L.gcase[lane] < 0 || !L.active[lane]) continue;
        const int k = m.new_of_bus[i];
        if (i == 0) {
            L.iters[lane] += 1;
            L.irs[lane] += nir;
        }
        if (k < 0) continue;
        const int g = lane / kLanes, l = lane % kLanes;
        const double d = L.x64[((long long)g * nbus + k) * kLanes + l];
        if (which == 0) {
            const double t = L.va[idx] + d;
            L.va[idx] = t;
            double co, s;
            if (fabs(d) <= kRotMax && L.lastmis[lane] > 1e3 * a.tol) {
                double sd, cd;
                small_sincos(d, &sd, &cd);
                co = L.cs[idx] * cd - L.sn[idx] * sd;
                s = L.sn[idx] * cd + L.cs[idx] * sd;
            } else {
                sincos(t, &s, &co);
            }
            L.cs[idx] = co;
            L.sn[idx] = s;
            L.e[idx] = L.vm[idx] * co;
            L.f[idx] = L.vm[idx] * s;
        } else {
            const double v = L.vm[idx] + d;
            L.vm[idx] = v;
            L.iv[idx] = 1.0 / v;
            L.e[idx] = v * L.cs[idx];
            L.f[idx] = v * L.sn[idx];
        }
    }
}

int grid_1d(long long total, int threads) {
    long long b = (total + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152LL * 64) b = 152LL * 64;
    return int(b);
}

template <class T, int W>
cudaError_t enqueue_pair(const LaneArgs &a, int nir, cudaStream_t s) {
    const LaneSet &L = a.L;
    const int nbus = a.dn.nbus;
    const int nmax = a.m0.n > a.m1.n ? a.m0.n : a.m1.n;
    const size_t smem = size_t(kStages) * kStageBytes + sizeof(T) * size_t(nmax) * W;
    cudaError_t e;
    for (int which = 0; which < 2; which++) {
        const DevMat &m = which ? a.m1 : a.m0;
        e = cudaMemsetAsync(L.nactive, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
        k_lane_mismatch<T><<<dim3((nbus + 7) / 8, L.ngroups), 256, 0, s>>>(a, which);
        k_lane_check<<<(L.ncp + 255) / 256, 256, 0, s>>>(a);
        k_lane_solve<T, W><<<L.ncp / W, kLaneThreads, smem, s>>>(a, which, 0);
        for (int k = 0; k < nir; k++) {
            k_lane_resid<T><<<dim3((m.n + 7) / 8, L.ngroups), 256, 0, s>>>(a, which);
            k_lane_solve<T, W><<<L.ncp / W, kLaneThreads, smem, s>>>(a, which, 1);
        }
        k_lane_update<<<grid_1d((long long)nbus * L.ncp, 256), 256, 0, s>>>(a, which, nir);
    }
    return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------ launchers

// Cases per solve group: the largest of 4, 2, 1 whose vectors fit in shared
// memory next to the staging ring (0: none fits).
int lane_width(int nmax, int prec, size_t smem_optin) {
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    for (int W : {4, 2, 1})
        if (size_t(kStages) * kStageBytes + elt * size_t(nmax) * W + 2048 <= smem_optin) return W;
    return 0;
}

template <class T, int W>
cudaError_t lane_attr(size_t smem) {
    return cudaFuncSetAttribute(k_lane_solve<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

cudaError_t lane_run(const LaneRun &r, cudaStream_t s) {
    LaneArgs a;
    a.dn = r.dn;
    a.dc = r.dc;
    a.m0 = r.m0;
    a.m1 = r.m1;
    a.L = r.L;
    a.F0 = r.F0;
    a.F1 = r.F1;
    a.fs0 = r.fs0;
    a.fs1 = r.fs1;
    a.A0 = r.A0;
    a.A1 = r.A1;
    a.tol = r.o.tol;
    a.flat = r.o.flat_start;
    a.spin = r.o.spin_limit > 0 ? unsigned(r.o.spin_limit) : kDefaultSpin;
    const LaneSet &L = r.L;
    const long long tot = (long long)r.dn.nbus * L.ncp;
    const int nmax = r.m0.n > r.m1.n ? r.m0.n : r.m1.n;
    const int W = lane_width(nmax, r.prec, r.smem_optin);
    if (W == 0) return cudaErrorInvalidValue;
    const size_t smem = size_t(kStages) * kStageBytes +
                        (r.prec == PF_FP64 ? sizeof(double) : sizeof(float)) * size_t(nmax) * W;
    cudaError_t e = r.prec == PF_FP64
                        ? (W == 4 ? lane_attr<double, 4>(smem) : W == 2 ? lane_attr<double, 2>(smem) : lane_attr<double, 1>(smem))
                        : (W == 4 ? lane_attr<float, 4>(smem) : W == 2 ? lane_attr<float, 2>(smem) : lane_attr<float, 1>(smem));
    if (e != cudaSuccess) return e;
    auto enqueue = [&](cudaStream_t st) {
        if (r.prec == PF_FP64)
            return W == 4 ? enqueue_pair<double, 4>(a, 0, st) : W == 2 ? enqueue_pair<double, 2>(a, 0, st)
                                                                       : enqueue_pair<double, 1>(a, 0, st);
        const int nir = r.o.ir_max < 2 ? r.o.ir_max : 2;
        return W == 4 ? enqueue_pair<float, 4>(a, nir, st) : W == 2 ? enqueue_pair<float, 2>(a, nir, st)
                                                                    : enqueue_pair<float, 1>(a, nir, st);
    };
    // own-factor groups: interleave their lanes' factors
    if (L.nown > 0) {
        for (int which = 0; which < 2; which++) {
            const DevMat &m = which ? r.m1 : r.m0;
            const long long n = (long long)m.stride * kLanes * L.nown;
            if (r.prec == PF_FP64)
                k_lane_factors<double><<<grid_1d(n, 256), 256, 0, s>>>(
                    a, which, static_cast<double *>(which ? L.LF1 : L.LF0));
            else
                k_lane_factors<float><<<grid_1d(n, 256), 256, 0, s>>>(
                    a, which, static_cast<float *>(which ? L.LF1 : L.LF0));
        }
    }
    k_lane_load<<<grid_1d(tot, 256), 256, 0, s>>>(a, r.vm, r.va);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // one P/Q pair as a CUDA graph, replayed until no case is active
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (r.use_graph) {
        cudaStream_t cs;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return e;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue(cs);
            e = cudaStreamEndCapture(cs, &graph);
            if (e2 != cudaSuccess) e = e2;
        }
        cudaStreamDestroy(cs);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return e;
        }
    }
    int active = 1;
    for (int it = 0; it < r.o.max_iter && active > 0; it++) {
        e = r.use_graph ? cudaGraphLaunch(exec, s) : enqueue(s);
        if (e != cudaSuccess) break;
        e = cudaMemcpyAsync(&active, L.nactive, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    // final convergence check of cases still active after max_iter pairs
    e = cudaMemsetAsync(L.nactive, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        if (r.prec == PF_FP64)
            k_lane_mismatch<double><<<dim3((r.dn.nbus + 7) / 8, L.ngroups), 256, 0, s>>>(a, 0);
        else
            k_lane_mismatch<float><<<dim3((r.dn.nbus + 7) / 8, L.ngroups), 256, 0, s>>>(a, 0);
        k_lane_check<<<(L.ncp + 255) / 256, 256, 0, s>>>(a);
        k_lane_store<<<grid_1d(tot, 256), 256, 0, s>>>(a, r.vm, r.va, r.res);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace gbpf
