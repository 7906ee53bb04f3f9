// gbpf_host.cpp -- host side of libgbpf: input checks, the bus admittance
// pattern, the symbolic analysis (ordering, fill, elimination tree, levels,
// schedules) and the C ABI entry points that enqueue the device kernels.
//
// Symbolic analysis (Section II.B of arxiv 1811.02512):
//   ordering   exact minimum degree on the elimination graph, ties to the
//              smallest bus (the paper leaves the ordering open);
//   fill       struct(L) from row subtrees of the elimination tree -- the
//              same filled graph G+(A) that FormFilledGraph produces
//              (Section II.B.1);
//   etree      parent[i] = min { j > i : l_ji != 0 } (Section II.B.2),
//              computed with path-compressed ancestor links;
//   levels     level = 1 for leaves, 1 + max over children otherwise, which is
//              exactly the repeated leaf peeling of FormHierarchicalPartition
//              (Section II.B, Table I).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <set>
#include <utility>

#include "gbpf_internal.h"

using namespace gbpf;

namespace {

pf_status fail(pf_ctx *ctx, pf_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return st;
}

pf_status cuda_fail(pf_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

template <class T>
pf_status upload(pf_ctx *ctx, T **dst, const T *src, size_t count) {
    *dst = nullptr;
    size_t bytes = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMalloc((void **)dst, bytes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    ctx->allocations.push_back(*dst);
    if (count) {
        e = cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy H2D");
    }
    return PF_OK;
}

template <class T>
pf_status dalloc(pf_ctx *ctx, T **dst, size_t count) {
    *dst = nullptr;
    cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * (count ? count : 1));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    ctx->allocations.push_back(*dst);
    return PF_OK;
}

void dfree(pf_ctx *ctx, void *p) {
    if (!p) return;
    auto it = std::find(ctx->allocations.begin(), ctx->allocations.end(), p);
    if (it != ctx->allocations.end()) ctx->allocations.erase(it);
    cudaFree(p);
}

#define TRY(x)                              \
    do {                                    \
        pf_status _st = (x);                \
        if (_st != PF_OK) return _st;       \
    } while (0)

// Forgets the context's CUDA graph of a run (see run_device_work).
void drop_graph(pf_ctx *ctx) {
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
    ctx->gkey.clear();
    ctx->gkey_last.clear();
}

// Enqueues `launch` (which returns the cudaError_t of its launches) on stream
// s, counting `nlaunch` kernel launches of kind `kind`; with profiling on the
// launch is bracketed by CUDA events on the same stream.
template <class F>
cudaError_t counted(pf_ctx *ctx, int kind, int nlaunch, cudaStream_t s, F launch) {
    KernelStat &k = ctx->kstat[kind];
    cudaEvent_t a = nullptr, b = nullptr;
    if (ctx->profiling) {
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
            return cudaErrorMemoryAllocation;
        cudaEventRecord(a, s);
    }
    cudaError_t e = launch();
    if (ctx->profiling) {
        cudaEventRecord(b, s);
        k.pending.push_back({a, b});
    }
    if (e == cudaSuccess && !ctx->graph_capturing) k.launches += nlaunch;
    if (e == cudaSuccess && ctx->graph_capturing) ctx->glaunches[kind] += nlaunch;
    return e;
}

// Done-flag epoch of the factorisations captured in a CUDA graph: the graph
// clears the flags itself (a memset node) and always publishes this epoch,
// which direct factorisations never reach (they restart at 1 below it).
constexpr unsigned kGraphEpoch = 0xFFFFFFF0u;
// The same for the Jacobian flags of the Newton-Raphson fallback inside a
// graph: its factorisations publish kNrGraphEpoch + 1, + 2, ... (direct
// launches stay below 0xF0000000 + their count, nr_epochs).
constexpr unsigned kNrGraphEpoch = 0xFFFF0000u;
constexpr int kFallbackIters = 30;  // Newton-Raphson steps of the FDPF -> NR fallback

void drain_events(pf_ctx *ctx, KernelStat &k) {
    for (auto &pr : k.pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(pr.second) == cudaSuccess &&
            cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess)
            k.ms += ms;
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    k.pending.clear();
}

int ypos(const pf_ctx *ctx, int i, int j) {
    const int *b = ctx->col.data() + ctx->rowptr[i];
    const int *e = ctx->col.data() + ctx->rowptr[i + 1];
    const int *p = std::lower_bound(b, e, j);
    return (p != e && *p == j) ? int(p - ctx->col.data()) : -1;
}

// ---------------------------------------------------------------- ordering

// Exact minimum degree: an ordered set of (degree, vertex) picks the vertex
// with the fewest remaining neighbours, ties to the smallest index; the
// neighbourhood of the eliminated vertex becomes a clique.
std::vector<int> min_degree_order(int n, std::vector<std::vector<int>> adj) {
    std::set<std::pair<int, int>> ready;
    for (int v = 0; v < n; v++) ready.insert({int(adj[v].size()), v});
    std::vector<int> order;
    order.reserve(n);
    std::vector<int> merged;
    while (!ready.empty()) {
        int v = ready.begin()->second;
        ready.erase(ready.begin());
        order.push_back(v);
        const std::vector<int> nb = std::move(adj[v]);
        adj[v].clear();
        for (int u : nb) {
            ready.erase({int(adj[u].size()), u});
            merged.clear();
            std::set_union(adj[u].begin(), adj[u].end(), nb.begin(), nb.end(),
                           std::back_inserter(merged));
            merged.erase(std::remove_if(merged.begin(), merged.end(),
                                        [&](int w) { return w == u || w == v; }),
                         merged.end());
            adj[u].swap(merged);
            ready.insert({int(adj[u].size()), u});
        }
    }
    return order;
}

// ---------------------------------------------------------------- analysis


// Partitioned inverse of the narrow top [t0, n) of one matrix (tail form 3,
// see DevMat): the columns of L_TT with their rows' depths for
// k_tail_inverse, and the chunked gather lists of z_T = W c_T (row i: its
// descendants j) and x_T = W^T D^-1 z_T (row i: its ancestors).  Chunks hold
// at most cw entries, cw the smallest power of two from 8 whose partial sums
// and the top's vector fit the idle staging ring.  Leaves pf3 / pb3 empty
// (no form 3) when the top is too large for a dense inverse.
void build_tail_inverse(HostMat &H) {
    const int n = H.n, t0 = H.t0, nt = H.nt;
    auto clear = [&] {
        H.pf3.clear();
        H.pb3.clear();
        H.tw_nfe = H.tw_nbe = H.tw_ne = 0;
    };
    if (nt <= 0 || nt > kClTailMax) return clear();
    std::vector<int> par(nt), dep(nt);
    for (int it = 0; it < nt; it++) {
        const int j = t0 + it;
        par[it] = H.Cp[j] < H.Cp[j + 1] ? H.Cr[H.Cp[j]] - t0 : -1;  // the first row of column j
        if (par[it] >= nt || (par[it] >= 0 && par[it] <= it)) return clear();
    }
    int depmax = 0;
    for (int it = nt - 1; it >= 0; it--) {
        dep[it] = par[it] < 0 ? 0 : dep[par[it]] + 1;
        depmax = std::max(depmax, dep[it] + 1);
    }
    H.twcp.assign(nt + 1, 0);
    H.twcdep.clear();
    H.twcpos.clear();
    for (int it = 0; it < nt; it++) {
        const int j = t0 + it;
        for (int p = H.Cp[j]; p < H.Cp[j + 1]; p++) {
            const int i = H.Cr[p] - t0;
            if (i < 0 || i >= nt) return clear();
            H.twcdep.push_back(dep[i]);
            H.twcpos.push_back(H.offLc + p);
        }
        H.twcp[it + 1] = int(H.twcdep.size());
    }
    H.tw_ne = int(H.twcdep.size());
    if (tail_inverse_smem(nt, H.tw_ne, depmax) > kTailInvSmem) return clear();
    H.twpar = par;
    H.twdep = dep;
    H.tw_depmax = depmax;
    std::vector<std::vector<int>> fr(nt), br(nt);
    for (int jt = 0; jt < nt; jt++)
        for (int a = par[jt]; a >= 0; a = par[a]) {
            fr[a].push_back(jt);  // W(a, jt): a row-a entry of the forward gather
            br[jt].push_back(a);  // W(a, jt) / D(a): a row-jt entry of the backward gather
        }
    auto nchunks = [&](const std::vector<std::vector<int>> &rows, int cw) {
        int c = 0;
        for (const auto &r : rows) c += int((r.size() + size_t(cw) - 1) / size_t(cw));
        return c;
    };
    int cw = 8;
    while ((size_t(nt) + size_t(std::max(nchunks(fr, cw), nchunks(br, cw)))) * sizeof(double) >
           size_t(kRingStages) * kPieceBytes)
        cw *= 2;
    auto lists = [&](const std::vector<std::vector<int>> &rows, bool fwd, std::vector<int> &rp,
                     std::vector<int2> &ch, std::vector<int> &cj, std::vector<int> &src,
                     std::vector<int> *dsrc) {
        rp.assign(nt + 1, 0);
        ch.clear();
        cj.clear();
        src.clear();
        if (dsrc) dsrc->clear();
        for (int it = 0; it < nt; it++) {
            const auto &r = rows[it];
            for (size_t e0 = 0; e0 < r.size(); e0 += size_t(cw)) {
                const size_t e1 = std::min(r.size(), e0 + size_t(cw));
                ch.push_back(int2{int(cj.size()), int(cj.size() + (e1 - e0))});
                for (size_t e = e0; e < e1; e++) {
                    const int j = r[e];
                    cj.push_back(j);
                    src.push_back(fwd ? it * nt + j : j * nt + it);
                    if (dsrc) dsrc->push_back(t0 + j);
                }
            }
            rp[it + 1] = int(ch.size());
        }
    };
    lists(fr, true, H.twfr, H.twfc, H.twfj, H.twfs, nullptr);
    lists(br, false, H.twbr, H.twbc, H.twbj, H.twbs, &H.twbd);
    auto pad32 = [](int64_t v) { return int((v + 31) / 32 * 32); };
    H.tw_nfe = int(H.twfj.size());
    H.tw_nbe = int(H.twbj.size());
    H.tw_boff = pad32(std::max(1, H.tw_nfe));
    H.tw_stride = H.tw_boff + pad32(std::max(1, H.tw_nbe));
    for (auto *v : {&H.twfj, &H.twbj, &H.twfs, &H.twbs, &H.twbd})
        if (v->empty()) v->push_back(0);
    if (H.twfc.empty()) H.twfc.push_back(int2{0, 0});
    if (H.twbc.empty()) H.twbc.push_back(int2{0, 0});
    (void)n;
}

// Scatter tail of one matrix (see DevMat): the schedules, the gathered value
// layout and the sweeps' piece lists that use them (pf2, pb2).  Without a
// tail (no narrow level at the top, or more than 32767 tail rows) the lists
// stay empty and the sweeps use pf, pb.
template <class MakePieces, class RunEnds>
pf_status build_tail(pf_ctx *ctx, HostMat &H, MakePieces &make_pieces, RunEnds &set_run_ends) {
    const int n = H.n;
    int lt = H.nlev;
    while (lt > 0 && H.lvl_ptr[lt] - H.lvl_ptr[lt - 1] <= kNarrowRows) lt--;
    const int t0 = H.lvl_ptr[lt], nt = n - t0;
    H.pf2.clear();
    H.pb2.clear();
    H.t0 = t0;
    H.nt = 0;
    H.ntl = 0;
    if (nt <= 0 || nt > 32767) return PF_OK;  // 16-bit row indices in the slots
    H.nt = nt;
    H.ntl = H.nlev - lt;
    struct Upd {
        int tgt, src, pos;
    };
    auto schedule = [&](bool fwd, std::vector<int> &SK, std::vector<int> &SI, std::vector<int> &spos) {
        SK.assign(1, 0);
        SI.clear();
        spos.clear();
        std::vector<std::vector<Upd>> lane(32);
        for (int li = 0; li < H.ntl; li++) {
            const int l = fwd ? lt + li : H.nlev - 1 - li;
            for (auto &v : lane) v.clear();
            for (int j = H.lvl_ptr[l]; j < H.lvl_ptr[l + 1]; j++) {
                if (fwd) {
                    for (int p = H.Cp[j]; p < H.Cp[j + 1]; p++) {
                        const int i = H.Cr[p];
                        lane[(i - t0) & 31].push_back({i - t0, j - t0, H.offLc + p});
                    }
                } else {
                    for (int q = H.Fp[j]; q < H.Fp[j + 1]; q++) {
                        const int i = H.Fc[q];
                        if (i >= t0) lane[(i - t0) & 31].push_back({i - t0, j - t0, H.offLr + q});
                    }
                }
            }
            size_t K = 0;
            for (auto &v : lane) {
                std::sort(v.begin(), v.end(), [](const Upd &a, const Upd &b) {
                    return a.tgt != b.tgt ? a.tgt < b.tgt : a.src < b.src;
                });
                K = std::max(K, v.size());
            }
            for (size_t k = 0; k < K; k++)
                for (int ln = 0; ln < 32; ln++) {
                    if (k < lane[ln].size()) {
                        const Upd &u = lane[ln][k];
                        SI.push_back(u.tgt | (u.src << 16));
                        spos.push_back(u.pos);
                    } else {
                        SI.push_back(-1);
                        spos.push_back(-1);
                    }
                }
            SK.push_back(SK.back() + int(K));
        }
    };
    std::vector<int> posf, posb;
    schedule(true, H.SKf, H.SIf, posf);
    schedule(false, H.SKb, H.SIb, posb);
    // tail rows' entries in columns below t0 (a prefix of each CSR row)
    H.PPp.assign(n + 1, 0);
    H.PPc.clear();
    std::vector<int> posp;
    for (int r = 0; r < n; r++) {
        if (r >= t0)
            for (int q = H.Fp[r]; q < H.Fp[r + 1] && H.Fc[q] < t0; q++) {
                H.PPc.push_back(H.Fc[q]);
                posp.push_back(H.offLr + q);
            }
        H.PPp[r + 1] = int(H.PPc.size());
    }
    // tail factor: per target of the tail columns its A slot, column and the
    // first gather term from a tail column (terms are in CSR order, k ascending)
    H.ft_g0 = H.Cp[t0] + t0;
    H.ft_e0 = H.Cp[t0];
    H.ft_ng = (n + int(H.Lp[n])) - H.ft_g0;
    H.ft_ne = int(H.Lp[n]) - H.ft_e0;
    H.tapos.assign(std::max(1, H.ft_ng), 0);
    H.tcol.assign(std::max(1, H.ft_ng), 0);
    H.gsplit.assign(std::max(1, H.ft_ng), 0);
    for (int c = t0; c < n; c++)
        for (int t = 0; t <= H.Cp[c + 1] - H.Cp[c]; t++) {
            const int g = H.Cp[c] + c + t;
            const int k = g - H.ft_g0;
            H.tapos[k] = t == 0 ? c : H.offLc + H.Cp[c] + t - 1;
            H.tcol[k] = c;
            int q = H.gp[g];
            while (q < H.gp[g + 1] && H.gl[q].z < t0) q++;
            H.gsplit[k] = q;
        }
    // the tail terms, packed with 16-bit positions (the tail factor is only
    // used when the tail has fewer than 65,536 entries)
    H.tptr.assign(size_t(std::max(1, H.ft_ng)) + 1, 0);
    H.tterm.clear();
    H.ft_tmax = 0;
    if (H.ft_ne < 65536) {
        for (int k = 0; k < H.ft_ng; k++) {
            for (int q = H.gsplit[k]; q < H.gp[H.ft_g0 + k + 1]; q++) {
                const int4 e = H.gl[q];
                H.tterm.push_back(int2{(e.x - H.ft_e0) | ((e.y - H.ft_e0) << 16), e.z - t0});
            }
            H.tptr[k + 1] = int(H.tterm.size());
        }
        if (H.tterm.empty()) H.tterm.push_back(int2{0, 0});
        for (int l = H.nlev - H.ntl; l < H.nlev; l++) {
            const int kb = H.Cp[H.lvl_ptr[l]] + H.lvl_ptr[l] - H.ft_g0;
            const int ke = H.Cp[H.lvl_ptr[l + 1]] + H.lvl_ptr[l + 1] - H.ft_g0;
            H.ft_tmax = std::max(H.ft_tmax, H.tptr[ke] - H.tptr[kb]);
        }
    }
    // level table, per-target descriptors and warp tasks of the tail factor,
    // so that its level loop needs no dependent global loads.  Within a level
    // every target gets the smallest power of two of lanes G that leaves one
    // term to a lane (at most 32: a GB300 FP64 instruction costs its warp
    // the same for one lane as for 32, so a target's instructions are
    // 2 ceil(terms / G) + log2 G, least near G = terms); the level's targets are
    // reordered by (G, terms) descending and cut into tasks of 32 / G
    // consecutive targets of one G (a warp's work), listed by decreasing
    // cost (terms per lane) so that warps taking tasks round-robin balance.
    // tipos maps a target to its position in the reordered level.
    H.tlev.assign(size_t(2) * size_t(std::max(1, H.ntl)), int4{0, 0, 0, 0});
    H.tinfo.assign(size_t(std::max(1, H.ft_ng)), int4{0, 0, 0, 0});
    H.tipos.assign(size_t(std::max(1, H.ft_ng)), 0);
    H.ttask.clear();
    H.ft_kmax = 0;
    if (H.ft_ne < 65536) {
        for (int li = 0; li < H.ntl; li++) {
            const int l = H.nlev - H.ntl + li;
            const int cb = H.lvl_ptr[l], ce = H.lvl_ptr[l + 1];
            const int kb = H.Cp[cb] + cb - H.ft_g0, ke = H.Cp[ce] + ce - H.ft_g0;
            const int tb = H.tptr[kb], te = H.tptr[ke];
            struct Tg {
                int G, cnt, k;
            };
            std::vector<Tg> ord;
            for (int k = kb; k < ke; k++) {
                const int cnt = H.tptr[k + 1] - H.tptr[k];
                int G = 1;
                while (G < 32 && cnt > G) G *= 2;
                ord.push_back(Tg{G, cnt, k});
            }
            std::sort(ord.begin(), ord.end(), [](const Tg &a, const Tg &b) {
                if (a.G != b.G) return a.G > b.G;
                if (a.cnt != b.cnt) return a.cnt > b.cnt;
                return a.k < b.k;
            });
            const int nk = ke - kb;
            std::vector<int4> tasks;  // {first position, targets, G, cost}
            for (int p = 0; p < nk;) {
                const int G = ord[size_t(p)].G;
                int q = p, cost = 0;
                while (q < nk && q - p < 32 / G && ord[size_t(q)].G == G) {
                    cost = std::max(cost, (ord[size_t(q)].cnt + G - 1) / G);
                    q++;
                }
                tasks.push_back(int4{p, q - p, G, cost});
                p = q;
            }
            std::stable_sort(tasks.begin(), tasks.end(), [](const int4 &a, const int4 &b) { return a.w > b.w; });
            const int t_first = int(H.ttask.size());
            for (const int4 &t : tasks) H.ttask.push_back(int4{t.x, t.y, t.z, 0});
            H.tlev[2 * li] = int4{kb, ke, tb, te};
            H.tlev[2 * li + 1] = int4{cb - t0, ce - t0, t_first, int(H.ttask.size())};
            H.ft_kmax = std::max(H.ft_kmax, nk);
            for (int p = 0; p < nk; p++) {
                const int k = ord[size_t(p)].k;
                const int c = H.tcol[k];
                const int t = k - (H.Cp[c] + c - H.ft_g0);
                H.tinfo[size_t(kb + p)] = int4{H.tptr[k] - tb, H.tptr[k + 1] - tb,
                                               t > 0 ? H.Cp[c] + t - 1 - H.ft_e0 : -1, c - t0};
                H.tipos[size_t(k)] = kb + p;
            }
        }
    }
    if (H.ttask.empty()) H.ttask.push_back(int4{0, 0, 1, 0});
    auto pad32 = [](int64_t v) { return int((v + 31) / 32 * 32); };
    H.tv_f = 0;
    H.tv_b = pad32(int64_t(posf.size()));
    H.tv_p = H.tv_b + pad32(int64_t(posb.size()));
    H.tv_stride = H.tv_p + pad32(int64_t(posp.size()));
    H.TVsrc.assign(std::max(1, H.tv_stride), -1);
    std::copy(posf.begin(), posf.end(), H.TVsrc.begin() + H.tv_f);
    std::copy(posb.begin(), posb.end(), H.TVsrc.begin() + H.tv_b);
    std::copy(posp.begin(), posp.end(), H.TVsrc.begin() + H.tv_p);
    const int budget = kPieceBytes - kPieceSlack;
    // scatter pieces: consecutive slot rows, 4 bytes of index and up to 8 of
    // value per slot, plus the slot-row offsets of the levels touched
    auto scatter_pieces = [&](const std::vector<int> &SK, std::vector<Piece> &out) {
        const int per = (budget - 64) / (32 * 12) - 1;  // slot rows per piece
        const int nrows = SK.back();
        int lv = 0;
        for (int k0 = 0; k0 < nrows;) {
            const int k1 = std::min(nrows, k0 + per);
            while (SK[lv + 1] <= k0) lv++;
            int lv1 = lv;
            while (lv1 < H.ntl && SK[lv1] < k1) lv1++;
            if (4 * (lv1 - lv + 8) + 12 * 32 * (k1 - k0) > budget)
                return fail(ctx, PF_ERR_ARG, "internal: scatter piece exceeds a stage");
            out.push_back(Piece{lv, lv1, k0 * 32, k1 * 32, 4, 0, t0, 0});
            k0 = k1;
        }
        return PF_OK;
    };
    // block-wide pieces over the tail rows: ptr gives the entries of a row
    auto row_pieces = [&](const std::vector<int> &ptr, int mode, int ebytes, int rbytes,
                          std::vector<Piece> &out) {
        int r = t0;
        while (r < n) {
            const int r0 = r;
            int64_t bytes = 16;
            while (r < n) {
                const int64_t rb = rbytes + int64_t(ebytes) * (ptr[r + 1] - ptr[r]);
                if (16 + rb > budget) return fail(ctx, PF_ERR_ARG, "internal: tail row exceeds a stage");
                if (r > r0 && bytes + rb > budget) break;
                bytes += rb;
                r++;
            }
            out.push_back(Piece{r0, r, ptr[r0], ptr[r], mode, 0, 0, 0});
        }
        return PF_OK;
    };
    std::vector<Piece> wide;
    // forward: wide levels, entries below the tail, scatter over the tail
    TRY(make_pieces(H.Fp, true, 12, 12, wide, lt));
    H.pf2 = wide;
    TRY(row_pieces(H.PPp, 5, 12, 12, H.pf2));
    H.pf3 = H.pf2;
    TRY(scatter_pieces(H.SKf, H.pf2));
    // backward: inverse diagonal of the tail rows, scatter, wide levels
    std::vector<int> zp(n + 1, 0);
    TRY(row_pieces(zp, 6, 12, 12, H.pb2));
    TRY(scatter_pieces(H.SKb, H.pb2));
    TRY(make_pieces(H.Cp, false, 12, 12, wide, lt));
    H.pb2.insert(H.pb2.end(), wide.begin(), wide.end());
    H.pb3 = wide;
    set_run_ends(H.pf2);
    set_run_ends(H.pb2);
    set_run_ends(H.pf3);
    set_run_ends(H.pb3);
    build_tail_inverse(H);
    return PF_OK;
}

// Device layout of one analysed matrix in level order (see DevMat).
pf_status build_layout(pf_ctx *ctx, HostMat &H) {
    const int n = H.n;
    const int64_t nnz = H.Lp[n];
    // level order: steps sorted by (level, step)
    H.lvl_ptr.assign(H.nlev + 1, 0);
    for (int j = 0; j < n; j++) H.lvl_ptr[H.level[j]]++;
    for (int l = 0; l < H.nlev; l++) H.lvl_ptr[l + 1] += H.lvl_ptr[l];
    H.neword.assign(n, 0);
    H.new_of_step.assign(n, 0);
    {
        std::vector<int> f(H.lvl_ptr.begin(), H.lvl_ptr.end() - 1);
        for (int j = 0; j < n; j++) {
            int r = f[H.level[j] - 1]++;
            H.neword[r] = j;
            H.new_of_step[j] = r;
        }
    }
    H.bus_new.assign(n, 0);
    H.local_new.assign(n, 0);
    H.new_of_bus.assign(ctx->nbus, -1);
    for (int r = 0; r < n; r++) {
        H.local_new[r] = H.perm[H.neword[r]];
        H.bus_new[r] = H.bus[H.local_new[r]];
        H.new_of_bus[H.bus_new[r]] = r;
    }
    // CSC in level order, rows ascending
    H.Cp.assign(n + 1, 0);
    for (int c = 0; c < n; c++) {
        int s = H.neword[c];
        H.Cp[c + 1] = H.Cp[c] + int(H.Lp[s + 1] - H.Lp[s]);
    }
    H.Cr.assign(nnz, 0);
    H.csc_of_steppos.assign(nnz, 0);
    {
        std::vector<std::pair<int, int>> tmp;
        for (int c = 0; c < n; c++) {
            int s = H.neword[c];
            tmp.clear();
            for (int64_t p = H.Lp[s]; p < H.Lp[s + 1]; p++)
                tmp.push_back({H.new_of_step[H.Li[p]], int(p)});
            std::sort(tmp.begin(), tmp.end());
            for (size_t t = 0; t < tmp.size(); t++) {
                H.Cr[H.Cp[c] + t] = tmp[t].first;
                H.csc_of_steppos[tmp[t].second] = H.Cp[c] + int(t);
                if (tmp[t].first <= c)
                    return fail(ctx, PF_ERR_ARG, "internal: level order is not triangular");
            }
        }
    }
    // CSR in level order (columns ascending, as c is visited ascending)
    H.Fp.assign(n + 1, 0);
    for (int64_t p = 0; p < nnz; p++) H.Fp[H.Cr[p] + 1]++;
    for (int r = 0; r < n; r++) H.Fp[r + 1] += H.Fp[r];
    H.Fc.assign(nnz, 0);
    H.Fpos.assign(nnz, 0);
    {
        std::vector<int> f(H.Fp.begin(), H.Fp.end() - 1);
        for (int c = 0; c < n; c++)
            for (int p = H.Cp[c]; p < H.Cp[c + 1]; p++) {
                int q = f[H.Cr[p]]++;
                H.Fc[q] = c;
                H.Fpos[q] = p;
            }
    }
    // update maps of the left-looking factor: CSR entry (c, k) updates column
    // c from the entries of column k at rows >= c (a contiguous tail of k)
    H.uoff.assign(nnz + 1, 0);
    for (int c = 0; c < n; c++)
        for (int q = H.Fp[c]; q < H.Fp[c + 1]; q++) {
            int k = H.Fc[q];
            H.uoff[q + 1] = H.uoff[q] + (H.Cp[k + 1] - H.Fpos[q]);
        }
    H.nupd = H.uoff[nnz];
    H.umap.assign(std::max<int64_t>(1, H.nupd), 0);
    for (int c = 0; c < n; c++) {
        const int *cb = H.Cr.data() + H.Cp[c];
        const int *ce = H.Cr.data() + H.Cp[c + 1];
        for (int q = H.Fp[c]; q < H.Fp[c + 1]; q++) {
            int k = H.Fc[q];
            int o = H.uoff[q];
            for (int p = H.Fpos[q]; p < H.Cp[k + 1]; p++) {
                int i = H.Cr[p];
                int tgt = 0;
                if (i != c) {
                    const int *f = std::lower_bound(cb, ce, i);
                    if (f == ce || *f != i) return fail(ctx, PF_ERR_ARG, "internal: fill not closed");
                    tgt = 1 + int(f - cb);
                }
                H.umap[o++] = tgt;
            }
        }
    }
    // gather lists of the same updates, grouped by target, in CSR-entry order
    H.gp.assign(size_t(n) + nnz + 1, 0);
    for (int c = 0; c < n; c++)
        for (int q = H.Fp[c]; q < H.Fp[c + 1]; q++) {
            const int k = H.Fc[q];
            for (int o = H.uoff[q], p = H.Fpos[q]; p < H.Cp[k + 1]; p++, o++)
                H.gp[size_t(H.Cp[c]) + c + H.umap[o] + 1]++;
        }
    for (size_t g = 0; g + 1 < H.gp.size(); g++) H.gp[g + 1] += H.gp[g];
    H.gl.assign(std::max<int64_t>(1, H.nupd), int4{0, 0, 0, 0});
    {
        std::vector<int> f(H.gp.begin(), H.gp.end() - 1);
        for (int c = 0; c < n; c++)
            for (int q = H.Fp[c]; q < H.Fp[c + 1]; q++) {
                const int k = H.Fc[q];
                for (int o = H.uoff[q], p = H.Fpos[q]; p < H.Cp[k + 1]; p++, o++)
                    H.gl[f[size_t(H.Cp[c]) + c + H.umap[o]]++] = int4{p, H.Fpos[q], k, 0};
            }
    }
    H.Cpos.assign(std::max<int64_t>(1, nnz), 0);
    for (int64_t q = 0; q < nnz; q++) H.Cpos[H.Fpos[q]] = int(q);
    auto pad32 = [](int64_t v) { return int((v + 31) / 32 * 32); };
    H.offDi = pad32(n);
    H.offLc = H.offDi + pad32(n);
    H.offLr = H.offLc + pad32(nnz);
    H.stride = H.offLr + pad32(nnz);
    // slot sources from the Ybus pattern
    H.src.assign(n + nnz, -1);
    for (int r = 0; r < n; r++) H.src[r] = ypos(ctx, H.bus_new[r], H.bus_new[r]);
    for (int c = 0; c < n; c++)
        for (int p = H.Cp[c]; p < H.Cp[c + 1]; p++)
            H.src[n + p] = ypos(ctx, H.bus_new[H.Cr[p]], H.bus_new[c]);
    H.br_slot.assign(3 * size_t(ctx->nbr), -1);
    for (int e = 0; e < ctx->nbr; e++) {
        int a = H.new_of_bus[ctx->branch[e].from], b = H.new_of_bus[ctx->branch[e].to];
        H.br_slot[3 * e + 0] = a;
        H.br_slot[3 * e + 1] = b;
        if (a >= 0 && b >= 0) {
            int lo = std::min(a, b), hi = std::max(a, b);
            const int *cb = H.Cr.data() + H.Cp[lo];
            const int *ce = H.Cr.data() + H.Cp[lo + 1];
            const int *f = std::lower_bound(cb, ce, hi);
            if (f == ce || *f != hi) return fail(ctx, PF_ERR_ARG, "internal: branch slot missing");
            H.br_slot[3 * e + 2] = H.offLc + int(f - H.Cr.data());
        }
    }
    // staged pieces: runs of rows (columns) of one level whose pointers,
    // indices and (8-byte) values fit one stage
    // staged pieces: runs of rows (columns) of one level, or whole narrow
    // levels, whose pointers, indices and values fit one stage; ebytes and
    // rbytes are the staged bytes per entry and per row
    auto make_pieces = [&](const std::vector<int> &ptr, bool ascending, int ebytes, int rbytes,
                           std::vector<Piece> &out, int nlev_used) {
        out.clear();
        const int budget = kPieceBytes - kPieceSlack;
        auto row_bytes = [&](int r) { return int64_t(rbytes) + int64_t(ebytes) * (ptr[r + 1] - ptr[r]); };
        auto level_bytes = [&](int l) {
            int64_t b = 4;  // its level pointer
            for (int r = H.lvl_ptr[l]; r < H.lvl_ptr[l + 1]; r++) b += row_bytes(r);
            return b;
        };
        auto split_rows = [&](int l, int mode) {  // one level in row runs
            int r = H.lvl_ptr[l], rend = H.lvl_ptr[l + 1];
            while (r < rend) {
                if (12 + row_bytes(r) > budget) {
                    // a row longer than one stage: consecutive parts of its entries
                    const int per = int((budget - 12 - rbytes - 32) / ebytes);
                    for (int e = ptr[r]; e < ptr[r + 1]; e += per)
                        out.push_back(Piece{r, r + 1, e, std::min(ptr[r + 1], e + per), 3, 0, l, l});
                    r++;
                    continue;
                }
                int r0 = r;
                int64_t bytes = 8 + 4;
                while (r < rend) {
                    if (r > r0 && bytes + row_bytes(r) > budget) break;
                    if (12 + row_bytes(r) > budget) break;
                    bytes += row_bytes(r);
                    r++;
                }
                out.push_back(Piece{r0, r, ptr[r0], ptr[r], mode, 0, l, l});
            }
            return true;
        };
        int li = 0;
        while (li < nlev_used) {
            int l = ascending ? li : nlev_used - 1 - li;
            const int lrows = H.lvl_ptr[l + 1] - H.lvl_ptr[l];
            if (lrows <= kNarrowRows) {
                int64_t bytes = 8 + level_bytes(l);
                if (bytes > budget) {  // a narrow level too large for one stage
                    if (!split_rows(l, 2)) return fail(ctx, PF_ERR_ARG, "internal: row exceeds a stage");
                    li++;
                    continue;
                }
                // whole narrow levels, as many consecutive ones as fit
                int lo = l, hi = l;
                li++;
                while (li < nlev_used) {
                    int l2 = ascending ? li : nlev_used - 1 - li;
                    if (H.lvl_ptr[l2 + 1] - H.lvl_ptr[l2] > kNarrowRows) break;
                    int64_t add = level_bytes(l2);
                    if (bytes + add > budget) break;
                    bytes += add;
                    lo = std::min(lo, l2);
                    hi = std::max(hi, l2);
                    li++;
                }
                const int r0 = H.lvl_ptr[lo], r1 = H.lvl_ptr[hi + 1];
                out.push_back(Piece{r0, r1, ptr[r0], ptr[r1], 2, 0, lo, hi});
                continue;
            }
            if (!split_rows(l, lrows <= 4 * kSweepWarps ? 1 : 0))
                return fail(ctx, PF_ERR_ARG, "internal: row exceeds a stage");
            li++;
        }
        return PF_OK;
    };
    // end of every run of single-warp pieces (modes 2, 3, 4)
    auto set_run_ends = [](std::vector<Piece> &out) {
        auto single = [](int mode) { return mode >= 2 && mode <= 4; };
        const int np = int(out.size());
        for (int j = np - 1; j >= 0; j--)
            if (single(out[j].mode))
                out[j].run_end = (j + 1 < np && single(out[j + 1].mode)) ? out[j + 1].run_end : j + 1;
    };
    // off-diagonal pattern of A by row, both triangles, fill excluded
    {
        std::vector<std::vector<std::pair<int, int>>> rowsA(n);
        for (int c = 0; c < n; c++)
            for (int p = H.Cp[c]; p < H.Cp[c + 1]; p++)
                if (H.src[n + p] >= 0) {
                    rowsA[H.Cr[p]].push_back({c, H.offLc + p});
                    rowsA[c].push_back({H.Cr[p], H.offLc + p});
                }
        H.Ap.assign(n + 1, 0);
        H.Aj.clear();
        H.Apos.clear();
        for (int r = 0; r < n; r++) {
            std::sort(rowsA[r].begin(), rowsA[r].end());
            for (auto &e : rowsA[r]) {
                H.Aj.push_back(e.first);
                H.Apos.push_back(e.second);
            }
            H.Ap[r + 1] = int(H.Aj.size());
        }
    }
    TRY(make_pieces(H.Fp, true, 12, 12, H.pf, H.nlev));
    TRY(make_pieces(H.Cp, false, 12, 12, H.pb, H.nlev));
    set_run_ends(H.pf);
    set_run_ends(H.pb);
    TRY(build_tail(ctx, H, make_pieces, set_run_ends));
    // Newton-Raphson Jacobian on the same pattern: 2 x 2 blocks (36 staged
    // bytes per FP64 block entry and per row), transposed slot sources, and
    // the block value layout [D | Dinv | Lc | Uc | Lr | Ur]
    TRY(make_pieces(H.Fp, true, 36, 36, H.pfJ, H.nlev));
    TRY(make_pieces(H.Cp, false, 36, 36, H.pbJ, H.nlev));
    set_run_ends(H.pfJ);
    set_run_ends(H.pbJ);
    H.srcT.assign(nnz, -1);
    for (int c = 0; c < n; c++)
        for (int p = H.Cp[c]; p < H.Cp[c + 1]; p++) H.srcT[p] = ypos(ctx, H.bus_new[c], H.bus_new[H.Cr[p]]);
    H.jD = 0;
    H.jDi = pad32(4 * int64_t(n));
    H.jLc = H.jDi + pad32(4 * int64_t(n));
    H.jUc = H.jLc + pad32(4 * nnz);
    H.jLr = H.jUc + pad32(4 * nnz);
    H.jUr = H.jLr + pad32(4 * nnz);
    H.jstride = H.jUr + pad32(4 * nnz);
    return PF_OK;
}

pf_status analyze_matrix(pf_ctx *ctx, int which, HostMat &H) {
    const int nbus = ctx->nbus;
    H = HostMat();
    for (int i = 0; i < nbus; i++) {
        int t = ctx->bus[i].type;
        bool in = (which == PF_MAT_BP) ? (t != PF_BUS_SLACK) : (t == PF_BUS_PQ);
        if (in) H.bus.push_back(i);
    }
    const int n = int(H.bus.size());
    H.n = n;
    std::vector<int> loc(nbus, -1);
    for (int a = 0; a < n; a++) loc[H.bus[a]] = a;
    std::vector<std::vector<int>> g(n);
    for (int a = 0; a < n; a++) {
        int i = H.bus[a];
        for (int p = ctx->rowptr[i]; p < ctx->rowptr[i + 1]; p++) {
            int j = ctx->col[p];
            if (j != i && loc[j] >= 0) g[a].push_back(loc[j]);
        }
    }
    H.perm = min_degree_order(n, g);
    H.iperm.assign(n, 0);
    for (int k = 0; k < n; k++) H.iperm[H.perm[k]] = k;
    // permuted graph
    std::vector<std::vector<int>> pg(n);
    for (int k = 0; k < n; k++) {
        for (int a : g[H.perm[k]]) pg[k].push_back(H.iperm[a]);
        std::sort(pg[k].begin(), pg[k].end());
    }
    // elimination tree with path-compressed ancestors
    H.parent.assign(n, -1);
    std::vector<int> anc(n, -1);
    for (int i = 0; i < n; i++)
        for (int k : pg[i]) {
            if (k >= i) break;
            int r = k;
            while (r != -1 && r != i) {
                int nx = anc[r];
                anc[r] = i;
                if (nx == -1) H.parent[r] = i;
                r = nx;
            }
        }
    // row patterns of L: union of etree paths from struct(A_i, < i) up to i
    std::vector<std::vector<int>> rows(n);
    std::vector<int> mark(n, -1);
    for (int i = 0; i < n; i++) {
        mark[i] = i;
        for (int k : pg[i]) {
            if (k >= i) break;
            for (int r = k; mark[r] != i; r = H.parent[r]) {
                rows[i].push_back(r);
                mark[r] = i;
            }
        }
        std::sort(rows[i].begin(), rows[i].end());
    }
    // columns of L (rows ascending because i is visited ascending)
    std::vector<int64_t> cnt(n + 1, 0);
    for (int i = 0; i < n; i++)
        for (int k : rows[i]) cnt[k + 1]++;
    H.Lp.assign(n + 1, 0);
    for (int k = 0; k < n; k++) H.Lp[k + 1] = H.Lp[k] + cnt[k + 1];
    const int64_t nnz_l = H.Lp[n];
    if (nnz_l > INT32_MAX / 2) return fail(ctx, PF_ERR_OOM, "factor too large (%lld)", (long long)nnz_l);
    H.Li.assign(nnz_l, 0);
    std::vector<int64_t> fill(H.Lp.begin(), H.Lp.end() - 1);
    for (int i = 0; i < n; i++)
        for (int k : rows[i]) H.Li[fill[k]++] = i;
    H.max_col = 0;
    for (int k = 0; k < n; k++) H.max_col = std::max<int>(H.max_col, int(H.Lp[k + 1] - H.Lp[k]));
    // levels: leaves 1, parents 1 + max over children
    H.level.assign(n, 1);
    for (int j = 0; j < n; j++)
        if (H.parent[j] >= 0) H.level[H.parent[j]] = std::max(H.level[H.parent[j]], H.level[j] + 1);
    H.nlev = 0;
    for (int j = 0; j < n; j++) H.nlev = std::max(H.nlev, H.level[j]);
    return build_layout(ctx, H);
}

// Program of the cluster engine for matrix `which` (see ClMat).  The
// elimination forest is cut into a top set T, closed under taking parents
// (it starts as the narrow tail of the tree), and the subtrees hanging below
// it.  Each subtree belongs wholly to one CTA, so its levels need only the
// CTA's own barrier and read only the CTA's own vector words; subtrees go to
// the least-loaded CTA, largest first, after the root of any subtree heavier
// than half a CTA's share has been moved into T (its children become
// subtrees).  Weight of a row: entries of its row and of its column of L,
// plus one.  T is solved through the inverse of its block of L (three
// cluster-wide steps); its rows go to the least-loaded CTA, heaviest first.
// A CTA's steps: its forward subtree levels (leaves have no entries), a
// cluster barrier, T's c = b - L_TB z_B, z = W c and x = W^T D^-1 z (each
// ending with a cluster barrier), its backward subtree levels, and a final
// cluster barrier.  Lanes per task: the smallest power of two that leaves at
// most four entries to a lane (at most 32).  A top set too large for the
// inverse leaves the program unusable (ok = 0).  Host only.
pf_status build_cluster(pf_ctx *ctx, int which, HostCl &P, int group) {
    const HostMat &H = ctx->hm[which];
    const int C = kClCtas, n = H.n, nbus = ctx->nbus;
    P = HostCl();
    P.rhsref.assign(nbus, -1);
    P.xref.assign(nbus, -1);
    P.tptr.assign(C + 1, 0);
    P.eptr.assign(C + 1, 0);
    P.vptr.assign(C + 1, 0);
    P.sptr.assign(C + 1, 0);
    if (n == 0) {
        P.ok = 1;
        P.tasks.assign(C, int4{0, 0, -1, 0});
        for (int r = 0; r <= C; r++) P.tptr[r] = r;
        P.max_tasks = 1;
        P.steps.push_back(int4{0, 0, 1, 0});
        P.refs.push_back(0);
        P.vsrc.push_back(int4{0, 0, 0, 0});
        return PF_OK;
    }
    auto rowlen = [&](int i) { return H.Fp[i + 1] - H.Fp[i]; };
    auto collen = [&](int i) { return H.Cp[i + 1] - H.Cp[i]; };
    std::vector<int> par(n);
    std::vector<std::vector<int>> kids(n);
    for (int j = 0; j < n; j++) {
        par[j] = collen(j) > 0 ? H.Cr[H.Cp[j]] : -1;
        if (par[j] >= 0) kids[par[j]].push_back(j);
    }
    std::vector<int64_t> sw(n);
    for (int j = 0; j < n; j++) sw[j] = rowlen(j) + collen(j) + 1;
    for (int j = 0; j < n; j++)
        if (par[j] >= 0) sw[par[j]] += sw[j];  // children come first in level order
    // top set: the narrow tail, then split roots
    std::vector<char> inT(n, 0);
    if (H.nt > 0)
        for (int i = H.t0; i < n; i++) inT[i] = 1;
    int64_t total = 0;
    for (int j = 0; j < n; j++)
        if (!inT[j]) total += rowlen(j) + collen(j) + 1;
    const int64_t share = (total + C - 1) / C;
    std::vector<int> roots;
    for (int j = 0; j < n; j++)
        if (!inT[j] && (par[j] < 0 || inT[par[j]])) roots.push_back(j);
    auto heavier = [&](int x, int y) { return sw[x] != sw[y] ? sw[x] < sw[y] : x > y; };
    std::make_heap(roots.begin(), roots.end(), heavier);
    while (!roots.empty() && 2 * sw[roots.front()] > share) {
        std::pop_heap(roots.begin(), roots.end(), heavier);
        const int r0 = roots.back();
        roots.pop_back();
        inT[r0] = 1;
        for (int c : kids[r0]) {
            roots.push_back(c);
            std::push_heap(roots.begin(), roots.end(), heavier);
        }
    }
    std::vector<int> &tnode = P.tnode;
    std::vector<int> trel(n, -1);
    for (int i = 0; i < n; i++)
        if (inT[i]) {
            trel[i] = int(tnode.size());
            tnode.push_back(i);
        }
    const int nt = int(tnode.size());
    P.nt = nt;
    // owners: subtrees by weight to the least-loaded CTA, T rows likewise
    std::vector<int> owner(n, 0);
    std::vector<int64_t> load(C, 0);
    std::sort(roots.begin(), roots.end(), [&](int x, int y) { return sw[x] != sw[y] ? sw[x] > sw[y] : x < y; });
    for (int r0 : roots) {
        const int r = int(std::min_element(load.begin(), load.end()) - load.begin());
        owner[r0] = r;
        load[r] += sw[r0];
    }
    for (int j = n - 1; j >= 0; j--)
        if (!inT[j] && par[j] >= 0 && !inT[par[j]]) owner[j] = owner[par[j]];
    P.bottom_load_max = *std::max_element(load.begin(), load.end());
    P.bottom_load_avg = total / C;
    // T: parents, the pattern of W = L_TT^-1 (it an ancestor of jt) by row and
    // by column, depths, and the columns of L_TT
    std::vector<std::vector<int>> wrow(nt), wcol(nt);
    if (nt > 0) {
        P.tpar.assign(nt, -1);
        for (int jt = 0; jt < nt; jt++) {
            const int pj = par[tnode[jt]];
            P.tpar[jt] = pj >= 0 ? trel[pj] : -1;
            if (pj >= 0 && (P.tpar[jt] < 0 || P.tpar[jt] <= jt)) return fail(ctx, PF_ERR_ARG, "internal: top set");
        }
        for (int jt = 0; jt < nt; jt++)
            for (int it = P.tpar[jt]; it >= 0; it = P.tpar[it]) {
                wrow[it].push_back(jt);
                wcol[jt].push_back(it);
            }
        for (auto &v : wrow) std::sort(v.begin(), v.end());
        P.tdepth.assign(nt, 0);
        for (int jt = nt - 1; jt >= 0; jt--)  // parents come after their children
            if (P.tpar[jt] >= 0) P.tdepth[jt] = P.tdepth[P.tpar[jt]] + 1;
        P.tdepth_max = 1 + *std::max_element(P.tdepth.begin(), P.tdepth.end());
        P.tcp.assign(nt + 1, 0);
        for (int jt = 0; jt < nt; jt++) {
            const int j = tnode[jt];
            for (int p = H.Cp[j]; p < H.Cp[j + 1]; p++) {
                if (!inT[H.Cr[p]]) return fail(ctx, PF_ERR_ARG, "internal: top set column");
                P.tcdep.push_back(P.tdepth[trel[H.Cr[p]]]);
                P.tcpos.push_back(H.offLc + p);
            }
            P.tcp[jt + 1] = int(P.tcdep.size());
        }
        if (P.tcdep.empty()) {
            P.tcdep.push_back(0);
            P.tcpos.push_back(0);
        }
        if (nt > kClTailMax || tail_inverse_smem(nt, P.tcp[nt], P.tdepth_max) > kTailInvSmem) return PF_OK;
        std::vector<int> ord(nt);
        std::vector<int64_t> wt(nt);
        for (int it = 0; it < nt; it++) {
            const int i = tnode[it];
            int below = 0;
            for (int q = H.Fp[i]; q < H.Fp[i + 1]; q++) below += !inT[H.Fc[q]];
            wt[it] = below + int64_t(wrow[it].size()) + int64_t(wcol[it].size()) + collen(i) + 1;
            ord[it] = it;
        }
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return wt[x] > wt[y]; });
        std::vector<int64_t> tl(C, 0);
        for (int it : ord) {
            const int r = int(std::min_element(tl.begin(), tl.end()) - tl.begin());
            owner[tnode[it]] = r;
            tl[r] += wt[it];
        }
    }
    // groups of subtree levels: a bottom row's group is its level / g; its
    // parent inside the group (-1: none), the paths up to the group's top
    const int g = std::max(1, std::min(group, kClGroupMax));
    P.group = g;
    std::vector<int> lev(n, 0);
    for (int l = 0; l < H.nlev; l++)
        for (int i = H.lvl_ptr[l]; i < H.lvl_ptr[l + 1]; i++) lev[i] = l;
    auto grp = [&](int i) { return lev[i] / g; };
    std::vector<int> gpar(n, -1);
    for (int j = 0; j < n; j++)
        if (!inT[j] && par[j] >= 0 && !inT[par[j]] && grp(par[j]) == grp(j)) gpar[j] = par[j];
    std::vector<std::vector<int>> gdesc(n), ganc(n);  // strict, inside the group
    for (int j = 0; j < n; j++)
        for (int a = gpar[j]; a >= 0; a = gpar[a]) {
            gdesc[a].push_back(j);
            ganc[j].push_back(a);  // nearest first
        }
    for (auto &v : gdesc) std::sort(v.begin(), v.end());
    std::vector<char> hasfwd(n, 0);
    for (int i = 0; i < n; i++)
        if (!inT[i]) hasfwd[i] = rowlen(i) > 0 || !gdesc[i].empty();
    // values of the groups' inverses: W(ganc[j][q-1], j) at GV index wbase[j] + q - 1
    std::vector<int> wbase(n, -1);
    P.gw_col.clear();
    P.gw_upd.clear();
    P.gv_info.clear();
    int ngv = 0;
    for (int j = 0; j < n; j++) {
        if (ganc[j].empty()) continue;
        const int Pn = 1 + int(ganc[j].size());
        wbase[j] = ngv;
        const int ub = int(P.gw_upd.size());
        std::vector<int> path(1, j);
        path.insert(path.end(), ganc[j].begin(), ganc[j].end());
        for (int pp = 0; pp + 1 < Pn; pp++) {
            const int m = path[size_t(pp)];
            for (int pos = H.Cp[m]; pos < H.Cp[m + 1]; pos++) {
                const int i = H.Cr[pos];
                for (int q = pp + 1; q < Pn; q++)
                    if (path[size_t(q)] == i) P.gw_upd.push_back(int4{pp, q, H.offLc + pos, 0});
            }
        }
        P.gw_col.push_back(int4{ub, int(P.gw_upd.size()), ngv, Pn});
        for (int q = 1; q < Pn; q++) P.gv_info.push_back(int4{0, path[size_t(q)], j, 0});
        ngv += Pn - 1;
    }
    P.n_gw = ngv;
    auto widx = [&](int a, int j) {  // GV index of W(a, j), a a strict ancestor of j in its group
        for (size_t q = 0; q < ganc[j].size(); q++)
            if (ganc[j][q] == a) return wbase[j] + int(q);
        return -1;
    };
    P.gm_ptr.assign(1, 0);
    P.gm_term.clear();
    int nm = 0;
    // a combined entry: a single identity term is the factor value itself
    // (kind 0), anything else a GV entry (kind 5) with its terms
    auto combined = [&](const std::vector<int2> &terms, int type, int i, int k) {
        if (terms.size() == 1 && terms[0].x < 0) return int4{0, terms[0].y, 0, 0};
        for (const int2 &t : terms) P.gm_term.push_back(t);
        P.gm_ptr.push_back(int(P.gm_term.size()));
        P.gv_info.push_back(int4{type, i, k, 0});
        return int4{5, P.n_gw + nm++, 0, 0};
    };
    // vector words: per bottom row b (its right-hand side, later its
    // solution) and z (its forward result, when it has a forward task); per
    // T row xb (right-hand side, then z), tc and tx
    std::vector<int> cnt(C, 0), xw(n, 0), zw(n, -1), tcw(std::max(1, nt), 0), txw(std::max(1, nt), 0);
    for (int i = 0; i < n; i++) {
        xw[i] = cnt[owner[i]]++;
        if (!inT[i] && hasfwd[i]) zw[i] = cnt[owner[i]]++;
    }
    for (int it = 0; it < nt; it++) {
        tcw[it] = cnt[owner[tnode[it]]]++;
        txw[it] = cnt[owner[tnode[it]]]++;
    }
    P.nx = *std::max_element(cnt.begin(), cnt.end());
    if (P.nx > 65535) return PF_OK;
    auto ref_xb = [&](int i) { return (owner[i] << 16) | xw[i]; };
    auto ref_z = [&](int i) { return (owner[i] << 16) | (!inT[i] && zw[i] >= 0 ? zw[i] : xw[i]); };
    auto ref_tc = [&](int i) { return (owner[i] << 16) | tcw[trel[i]]; };
    auto ref_tx = [&](int i) { return (owner[i] << 16) | txw[trel[i]]; };
    for (int i = 0; i < n; i++) {
        P.rhsref[H.bus_new[i]] = ref_xb(i);
        P.xref[H.bus_new[i]] = inT[i] ? ref_tx(i) : ref_xb(i);
    }
    // per CTA: its bottom rows by group
    int ngrp = 0;
    for (int i = 0; i < n; i++)
        if (!inT[i]) ngrp = std::max(ngrp, grp(i) + 1);
    std::vector<std::vector<std::vector<int>>> mine(C, std::vector<std::vector<int>>(std::max(1, ngrp)));
    for (int i = 0; i < n; i++)
        if (!inT[i]) mine[owner[i]][grp(i)].push_back(i);
    for (int r = 0; r < C; r++) {
        std::vector<int4> tasks, steps;
        std::vector<int> refs;
        std::vector<int4> esrc, dsrc;
        std::vector<int> dtask;  // tasks whose diagonal index needs the final entry count
        int maxlen = 0;
        auto add = [&](int out, int in, int dsrcpos) {
            tasks.push_back(int4{out, in, -1, int(refs.size())});
            if (dsrcpos >= 0) {
                tasks.back().z = int(dsrc.size());
                dtask.push_back(int(tasks.size()) - 1);
                dsrc.push_back(int4{0, dsrcpos, 0, 0});
            }
        };
        auto close = [&]() { maxlen = std::max(maxlen, int(refs.size()) - tasks.back().w); };
        // the tasks of a step (from tb on) by entry count, each task's own
        // entries unchanged: a warp's lanes then take tasks of one length
        // (an FP64 instruction costs its warp the same whatever number of
        // lanes it serves)
        auto sort_step = [&](int tb) {
            const int te = int(tasks.size());
            if (te - tb < 2) return;
            auto end_of = [&](int t) { return t + 1 < te ? tasks[t + 1].w : int(refs.size()); };
            std::vector<int> ord(te - tb);
            for (int k = 0; k < te - tb; k++) ord[k] = k;
            std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
                return end_of(tb + x) - tasks[tb + x].w < end_of(tb + y) - tasks[tb + y].w;
            });
            const int base = tasks[tb].w;
            std::vector<int4> nt_(te - tb), ne_;
            std::vector<int> nr_;
            std::vector<int> at(te - tb);
            for (int k = 0; k < te - tb; k++) {
                const int t = tb + ord[k];
                nt_[k] = tasks[t];
                nt_[k].w = base + int(nr_.size());
                nr_.insert(nr_.end(), refs.begin() + tasks[t].w, refs.begin() + end_of(t));
                ne_.insert(ne_.end(), esrc.begin() + tasks[t].w, esrc.begin() + end_of(t));
                at[ord[k]] = tb + k;
            }
            std::copy(nt_.begin(), nt_.end(), tasks.begin() + tb);
            std::copy(nr_.begin(), nr_.end(), refs.begin() + base);
            std::copy(ne_.begin(), ne_.end(), esrc.begin() + base);
            for (int &t : dtask)
                if (t >= tb) t = at[t - tb];
        };
        // a step over the tasks added since tb; cluster = 1: a cluster barrier follows
        auto step = [&](int tb, int cluster) {
            int G = 1;
            while (G < 32 && maxlen > 4 * G) G *= 2;
            steps.push_back(int4{tb, int(tasks.size()), G, cluster});
            maxlen = 0;
        };
        for (int G0 = 0; G0 < ngrp; G0++) {  // forward subtree groups
            const int tb = int(tasks.size());
            for (int i : mine[r][G0]) {
                if (!hasfwd[i]) continue;
                add(zw[i], xw[i], -1);
                for (int j : gdesc[i]) {  // - W(i, j) b_j
                    refs.push_back(ref_xb(j));
                    esrc.push_back(int4{3, widx(i, j), 0, 0});
                }
                std::map<int, std::vector<int2>> comb;  // k below the group -> terms W(i, j) L(j, k)
                std::vector<int> js(1, i);
                js.insert(js.end(), gdesc[i].begin(), gdesc[i].end());
                for (int j : js)
                    for (int q = H.Fp[j]; q < H.Fp[j + 1]; q++) {
                        const int k = H.Fc[q];
                        if (grp(k) < G0) comb[k].push_back(int2{j == i ? -1 : widx(i, j), H.offLr + q});
                    }
                for (auto &kv : comb) {
                    refs.push_back(ref_z(kv.first));
                    esrc.push_back(combined(kv.second, 1, i, kv.first));
                }
                close();
            }
            sort_step(tb);
            if (int(tasks.size()) > tb) step(tb, 0);
        }
        step(int(tasks.size()), 1);
        if (nt > 0) {
            for (int kind = 1; kind <= 3; kind++) {
                const int tb = int(tasks.size());
                for (int it = 0; it < nt; it++) {
                    const int i = tnode[it];
                    if (owner[i] != r) continue;
                    if (kind == 1) {  // c = b - L_TB z_B
                        add(tcw[it], xw[i], -1);
                        for (int q = H.Fp[i]; q < H.Fp[i + 1]; q++)
                            if (!inT[H.Fc[q]]) {
                                refs.push_back(ref_z(H.Fc[q]));
                                esrc.push_back(int4{0, H.offLr + q, 0, 0});
                            }
                    } else if (kind == 2) {  // z = W c
                        add(xw[i], tcw[it], -1);
                        for (int jt : wrow[it]) {
                            refs.push_back(ref_tc(tnode[jt]));
                            esrc.push_back(int4{1, it * nt + jt, 0, 0});
                        }
                    } else {  // x = W^T D^-1 z
                        add(txw[it], xw[i], H.offDi + i);
                        for (int at : wcol[it]) {
                            refs.push_back(ref_xb(tnode[at]));
                            esrc.push_back(int4{2, at * nt + it, H.offDi + tnode[at], 0});
                        }
                    }
                    close();
                }
                sort_step(tb);
                step(tb, 1);
            }
        }
        for (int G0 = ngrp - 1; G0 >= 0; G0--) {  // backward subtree groups
            const int tb = int(tasks.size());
            for (int i : mine[r][G0]) {
                add(xw[i], !inT[i] && zw[i] >= 0 ? zw[i] : xw[i], H.offDi + i);
                for (int a : ganc[i]) {  // - W(a, i) z_a / d_a
                    refs.push_back(ref_z(a));
                    esrc.push_back(int4{4, widx(a, i), H.offDi + a, 0});
                }
                std::map<int, std::vector<int2>> comb;  // k above the group -> terms W(j, i) L(k, j)
                std::vector<int> js(1, i);
                js.insert(js.end(), ganc[i].begin(), ganc[i].end());
                for (int j : js)
                    for (int pos = H.Cp[j]; pos < H.Cp[j + 1]; pos++) {
                        const int k = H.Cr[pos];
                        if (inT[k] || grp(k) > G0) comb[k].push_back(int2{j == i ? -1 : widx(j, i), H.offLc + pos});
                    }
                for (auto &kv : comb) {
                    refs.push_back(inT[kv.first] ? ref_tx(kv.first) : ref_xb(kv.first));
                    esrc.push_back(combined(kv.second, 2, i, kv.first));
                }
                close();
            }
            sort_step(tb);
            if (int(tasks.size()) > tb) step(tb, 0);
        }
        step(int(tasks.size()), 1);
        const int ne = int(refs.size());
        for (int t : dtask) tasks[t].z += ne;
        tasks.push_back(int4{0, 0, -1, ne});  // sentinel
        P.tptr[r + 1] = P.tptr[r] + int(tasks.size());
        P.eptr[r + 1] = P.eptr[r] + ne;
        P.vptr[r + 1] = P.vptr[r] + ne + int(dsrc.size());
        P.sptr[r + 1] = P.sptr[r] + int(steps.size());
        P.tasks.insert(P.tasks.end(), tasks.begin(), tasks.end());
        P.steps.insert(P.steps.end(), steps.begin(), steps.end());
        P.refs.insert(P.refs.end(), refs.begin(), refs.end());
        P.vsrc.insert(P.vsrc.end(), esrc.begin(), esrc.end());
        P.vsrc.insert(P.vsrc.end(), dsrc.begin(), dsrc.end());
        P.max_tasks = std::max(P.max_tasks, tasks.size());
        P.max_steps = std::max(P.max_steps, steps.size());
        P.max_e = std::max(P.max_e, size_t(ne));
        P.max_v = std::max(P.max_v, size_t(ne) + dsrc.size());
    }
    if (P.refs.empty()) P.refs.push_back(0);
    if (P.vsrc.empty()) P.vsrc.push_back(int4{0, 0, 0, 0});
    P.n_gm = nm;
    P.n_gwcol = int(P.gw_col.size());
    if (P.gw_col.empty()) P.gw_col.push_back(int4{0, 0, 0, 1});
    if (P.gw_upd.empty()) P.gw_upd.push_back(int4{0, 0, 0, 0});
    if (P.gm_term.empty()) P.gm_term.push_back(int2{-1, 0});
    P.ok = 1;
    return PF_OK;
}

// Dynamic shared memory of the cluster engine's CTA for both matrices'
// programs, and the byte offsets of their regions (16-byte aligned).
size_t cluster_smem_layout(pf_ctx *ctx) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 15) / 16 * 16;
        return int(o);
    };
    for (int w = 0; w < 2; w++) {
        const HostCl &P = ctx->hcl[w];
        ClMat &M = ctx->cl[w];
        M.so_x = take(sizeof(double) * std::max(1, P.nx));
        M.so_tasks = take(sizeof(int4) * std::max<size_t>(1, P.max_tasks));
        M.so_steps = take(sizeof(int4) * std::max<size_t>(1, P.max_steps));
        M.so_addr = take(sizeof(uint32_t) * std::max<size_t>(1, P.max_e));
        M.so_vals = take(sizeof(double) * std::max<size_t>(1, P.max_v));
    }
    return off;
}

// Uploads an int array padded by 16 bytes so that 16-byte-rounded bulk
// copies of its tail stay inside the allocation.
pf_status upload_padded(pf_ctx *ctx, int **dst, const std::vector<int> &v) {
    std::vector<int> tmp(v);
    tmp.resize(v.size() + 8, 0);
    return upload(ctx, dst, tmp.data(), tmp.size());
}

pf_status upload_cluster(pf_ctx *ctx, int w) {
    const HostCl &P = ctx->hcl[w];
    ClMat &M = ctx->cl[w];
    M.nt = P.nt;
    M.nval = int(P.vsrc.size());
    if (P.nt > 0) {
        TRY(upload_padded(ctx, &M.tpar, P.tpar));
        TRY(upload_padded(ctx, &M.tcp, P.tcp));
        TRY(upload_padded(ctx, &M.tcdep, P.tcdep));
        TRY(upload_padded(ctx, &M.tcpos, P.tcpos));
        TRY(upload_padded(ctx, &M.tdepth, P.tdepth));
        M.ntail_e = P.tcp[P.nt];
        M.tdepth_max = P.tdepth_max;
        TRY(dalloc(ctx, &ctx->clW[w], size_t(P.nt) * size_t(P.nt)));
    }
    TRY(upload(ctx, &M.vsrc, P.vsrc.data(), P.vsrc.size()));
    TRY(dalloc(ctx, &M.vals, P.vsrc.size()));
    TRY(upload(ctx, &M.tasks, P.tasks.data(), P.tasks.size()));
    TRY(upload_padded(ctx, &M.tptr, P.tptr));
    TRY(upload(ctx, &M.steps, P.steps.data(), P.steps.size()));
    TRY(upload_padded(ctx, &M.sptr, P.sptr));
    TRY(upload_padded(ctx, &M.refs, P.refs));
    TRY(upload_padded(ctx, &M.eptr, P.eptr));
    TRY(upload_padded(ctx, &M.vptr, P.vptr));
    TRY(upload_padded(ctx, &M.rhsref, P.rhsref));
    TRY(upload_padded(ctx, &M.xref, P.xref));
    M.n_gwcol = P.n_gwcol;
    M.n_gw = P.n_gw;
    M.n_gm = P.n_gm;
    TRY(upload(ctx, &M.gw_col, P.gw_col.data(), P.gw_col.size()));
    TRY(upload(ctx, &M.gw_upd, P.gw_upd.data(), P.gw_upd.size()));
    TRY(upload_padded(ctx, &M.gm_ptr, P.gm_ptr));
    TRY(upload(ctx, &M.gm_term, P.gm_term.data(), P.gm_term.size()));
    TRY(dalloc(ctx, &M.gv, size_t(std::max(1, P.n_gw + P.n_gm))));
    return PF_OK;
}

pf_status upload_matrix(pf_ctx *ctx, const HostMat &H, DevMat &D) {
    D.n = H.n;
    D.nnz = int(H.Lp[H.n]);
    D.nlev = H.nlev;
    D.max_col = H.max_col;
    D.nupd = H.nupd;
    D.offDi = H.offDi;
    D.offLc = H.offLc;
    D.offLr = H.offLr;
    D.stride = H.stride;
    D.npf = int(H.pf.size());
    D.npb = int(H.pb.size());
    TRY(upload_padded(ctx, &D.bus, H.bus_new));
    TRY(upload_padded(ctx, &D.local, H.local_new));
    TRY(upload_padded(ctx, &D.new_of_bus, H.new_of_bus));
    TRY(upload_padded(ctx, &D.lvl_ptr, H.lvl_ptr));
    TRY(upload_padded(ctx, &D.Cp, H.Cp));
    TRY(upload_padded(ctx, &D.Cr, H.Cr));
    TRY(upload_padded(ctx, &D.Fp, H.Fp));
    TRY(upload_padded(ctx, &D.Fc, H.Fc));
    TRY(upload_padded(ctx, &D.Fpos, H.Fpos));
    TRY(upload_padded(ctx, &D.uoff, H.uoff));
    TRY(upload_padded(ctx, &D.umap, H.umap));
    TRY(upload_padded(ctx, &D.gp, H.gp));
    TRY(upload(ctx, &D.gl, H.gl.data(), H.gl.size()));
    TRY(upload_padded(ctx, &D.Cpos, H.Cpos));
    TRY(upload_padded(ctx, &D.src, H.src));
    TRY(upload_padded(ctx, &D.br_slot, H.br_slot));
    TRY(upload_padded(ctx, &D.Ap, H.Ap));
    TRY(upload_padded(ctx, &D.Aj, H.Aj));
    TRY(upload_padded(ctx, &D.Apos, H.Apos));
    TRY(upload(ctx, &D.pfJ, H.pfJ.data(), H.pfJ.size()));
    TRY(upload(ctx, &D.pbJ, H.pbJ.data(), H.pbJ.size()));
    TRY(upload_padded(ctx, &D.srcT, H.srcT));
    D.npfJ = int(H.pfJ.size());
    D.npbJ = int(H.pbJ.size());
    D.jD = H.jD; D.jDi = H.jDi; D.jLc = H.jLc; D.jUc = H.jUc; D.jLr = H.jLr; D.jUr = H.jUr;
    D.jstride = H.jstride;
    TRY(upload(ctx, &D.pf, H.pf.data(), H.pf.size()));
    TRY(upload(ctx, &D.pb, H.pb.data(), H.pb.size()));
    D.t0 = H.t0;
    D.nt = H.nt;
    D.ntl = H.ntl;
    D.npf2 = int(H.pf2.size());
    D.npb2 = int(H.pb2.size());
    D.npf3 = D.npb3 = 0;
    if (H.nt > 0 && H.tw_ne > 0 && !H.pf3.empty() && !H.pb3.empty()) {
        TRY(upload(ctx, &D.pf3, H.pf3.data(), H.pf3.size()));
        TRY(upload(ctx, &D.pb3, H.pb3.data(), H.pb3.size()));
        TRY(upload(ctx, &D.twfc, H.twfc.data(), H.twfc.size()));
        TRY(upload(ctx, &D.twbc, H.twbc.data(), H.twbc.size()));
        TRY(upload_padded(ctx, &D.twfr, H.twfr));
        TRY(upload_padded(ctx, &D.twbr, H.twbr));
        TRY(upload_padded(ctx, &D.twfj, H.twfj));
        TRY(upload_padded(ctx, &D.twbj, H.twbj));
        TRY(upload_padded(ctx, &D.twfs, H.twfs));
        TRY(upload_padded(ctx, &D.twbs, H.twbs));
        TRY(upload_padded(ctx, &D.twbd, H.twbd));
        TRY(upload_padded(ctx, &D.twpar, H.twpar));
        TRY(upload_padded(ctx, &D.twcp, H.twcp));
        TRY(upload_padded(ctx, &D.twcdep, H.twcdep));
        TRY(upload_padded(ctx, &D.twcpos, H.twcpos));
        TRY(upload_padded(ctx, &D.twdep, H.twdep));
        D.npf3 = int(H.pf3.size());
        D.npb3 = int(H.pb3.size());
        D.tw_nfc = int(H.twfr.back());
        D.tw_nbc = int(H.twbr.back());
        D.tw_nfe = H.tw_nfe;
        D.tw_nbe = H.tw_nbe;
        D.tw_boff = H.tw_boff;
        D.tw_stride = H.tw_stride;
        D.tw_ne = H.tw_ne;
        D.tw_depmax = H.tw_depmax;
    }
    if (H.nt > 0) {
        TRY(upload(ctx, &D.pf2, H.pf2.data(), H.pf2.size()));
        TRY(upload(ctx, &D.pb2, H.pb2.data(), H.pb2.size()));
        TRY(upload_padded(ctx, &D.SKf, H.SKf));
        TRY(upload_padded(ctx, &D.SIf, H.SIf));
        TRY(upload_padded(ctx, &D.SKb, H.SKb));
        TRY(upload_padded(ctx, &D.SIb, H.SIb));
        TRY(upload_padded(ctx, &D.PPp, H.PPp));
        TRY(upload_padded(ctx, &D.PPc, H.PPc));
        TRY(upload_padded(ctx, &D.ZP, std::vector<int>(H.n + 1, 0)));
        TRY(upload_padded(ctx, &D.TVsrc, H.TVsrc));
        D.tv_f = H.tv_f;
        D.tv_b = H.tv_b;
        D.tv_p = H.tv_p;
        D.tv_stride = H.tv_stride;
        TRY(upload_padded(ctx, &D.tapos, H.tapos));
        TRY(upload_padded(ctx, &D.gsplit, H.gsplit));
        if (H.tterm.empty()) return fail(ctx, PF_ERR_ARG, "internal: tail terms");
        TRY(upload(ctx, &D.tterm, H.tterm.data(), H.tterm.size()));
        D.ft_tterms = int(H.tterm.size());
        TRY(upload(ctx, &D.tlev, H.tlev.data(), H.tlev.size()));
        TRY(upload(ctx, &D.tinfo, H.tinfo.data(), H.tinfo.size()));
        TRY(upload(ctx, &D.ttask, H.ttask.data(), H.ttask.size()));
        D.ft_ntask = int(H.ttask.size());
        TRY(upload_padded(ctx, &D.tipos, H.tipos));
        D.ft_kmax = H.ft_kmax;
        D.ft_tmax = H.ft_ne < 65536 ? H.ft_tmax : -1;
        D.ft_ng = H.ft_ng;
        D.ft_ne = H.ft_ne;
        D.ft_g0 = H.ft_g0;
        D.ft_e0 = H.ft_e0;
    }
    return PF_OK;
}

pf_status ensure_device(pf_ctx *ctx) {
    const int nbus = ctx->nbus, nbranch = ctx->nbr;
    const pf_bus *bus = ctx->bus.data();
    const pf_branch *branch = ctx->branch.data();
    if (ctx->on_device) return PF_OK;
    cudaError_t ce = cudaGetDevice(&ctx->device);
    if (ce != cudaSuccess) return cuda_fail(ctx, ce, "no CUDA device");
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    ctx->smem_optin = size_t(optin);
    int per_sm = 0;
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device);
    ctx->smem_per_sm = size_t(per_sm);

    // device network tables
    DevNet &dn = ctx->dn;
    dn.nbus = nbus;
    dn.nbr = nbranch;
    dn.nnz = ctx->rowptr[nbus];
    std::vector<int> btype(nbus), bf(nbranch), bt(nbranch), bst(nbranch);
    std::vector<double> pd(nbus), qd(nbus), gs(nbus), bs(nbus), pg(nbus), vs(nbus), va(nbus);
    std::vector<double> rr(nbranch), xx(nbranch), bb(nbranch), tp(nbranch);
    for (int i = 0; i < nbus; i++) {
        btype[i] = bus[i].type; pd[i] = bus[i].pd; qd[i] = bus[i].qd; gs[i] = bus[i].gs;
        bs[i] = bus[i].bs; pg[i] = bus[i].pg; vs[i] = bus[i].vset; va[i] = bus[i].va;
    }
    for (int e = 0; e < nbranch; e++) {
        bf[e] = branch[e].from; bt[e] = branch[e].to; bst[e] = branch[e].status;
        rr[e] = branch[e].r; xx[e] = branch[e].x; bb[e] = branch[e].b;
        tp[e] = branch[e].tap == 0.0 ? 1.0 : branch[e].tap;
    }
    const std::vector<int> &ydiag = ctx->ydiag, &inc_ptr = ctx->inc_ptr, &inc_br = ctx->inc_br,
                           &inc_side = ctx->inc_side, &inc_pos = ctx->inc_pos, &br_pos = ctx->br_pos;
    pf_status st = PF_OK;
    do {
        if ((st = upload(ctx, &dn.btype, btype.data(), nbus))) break;
        if ((st = upload(ctx, &dn.pd, pd.data(), nbus))) break;
        if ((st = upload(ctx, &dn.qd, qd.data(), nbus))) break;
        if ((st = upload(ctx, &dn.gs, gs.data(), nbus))) break;
        if ((st = upload(ctx, &dn.bs, bs.data(), nbus))) break;
        if ((st = upload(ctx, &dn.pg, pg.data(), nbus))) break;
        if ((st = upload(ctx, &dn.vset, vs.data(), nbus))) break;
        if ((st = upload(ctx, &dn.va0, va.data(), nbus))) break;
        if ((st = upload(ctx, &dn.bf, bf.data(), nbranch))) break;
        if ((st = upload(ctx, &dn.bt, bt.data(), nbranch))) break;
        if ((st = upload(ctx, &dn.bstatus, bst.data(), nbranch))) break;
        if ((st = upload(ctx, &dn.br, rr.data(), nbranch))) break;
        if ((st = upload(ctx, &dn.bx, xx.data(), nbranch))) break;
        if ((st = upload(ctx, &dn.bb, bb.data(), nbranch))) break;
        if ((st = upload(ctx, &dn.btap, tp.data(), nbranch))) break;
        if ((st = upload(ctx, &dn.rowptr, ctx->rowptr.data(), ctx->rowptr.size()))) break;
        if ((st = upload(ctx, &dn.col, ctx->col.data(), ctx->col.size()))) break;
        if ((st = upload(ctx, &dn.ydiag, ydiag.data(), ydiag.size()))) break;
        if ((st = upload(ctx, &dn.inc_ptr, inc_ptr.data(), inc_ptr.size()))) break;
        if ((st = upload(ctx, &dn.inc_br, inc_br.data(), inc_br.size()))) break;
        if ((st = upload(ctx, &dn.inc_side, inc_side.data(), inc_side.size()))) break;
        if ((st = upload(ctx, &dn.inc_pos, inc_pos.data(), inc_pos.size()))) break;
        if ((st = upload(ctx, &dn.br_pos, br_pos.data(), br_pos.size()))) break;
        dn.noff = int(ctx->yoff.size());
        if ((st = upload(ctx, &dn.yoff, ctx->yoff.data(), ctx->yoff.size()))) break;
        if ((st = upload(ctx, &dn.yoff_br, ctx->yoff_br.data(), ctx->yoff_br.size()))) break;
        if ((st = upload(ctx, &dn.mis_ord, ctx->mis_ord.data(), ctx->mis_ord.size()))) break;
        if ((st = upload(ctx, &dn.mis_ord_cl, ctx->mis_ord_cl.data(), ctx->mis_ord_cl.size()))) break;
        if ((st = dalloc(ctx, &dn.G, dn.nnz))) break;
        if ((st = dalloc(ctx, &dn.B, dn.nnz))) break;
        if ((st = dalloc(ctx, &dn.Bp, dn.nnz))) break;
    } while (0);
    if (st != PF_OK) return st;
    if (ctx->analyzed)
        for (int w = 0; w < 2; w++) TRY(upload_matrix(ctx, ctx->hm[w], ctx->dm[w]));
    ctx->on_device = true;
    return PF_OK;
}

pf_status ensure_cases(pf_ctx *ctx) {
    if (ctx->dc.ncase > 0) return PF_OK;
    return pf_set_cases(ctx, 1, nullptr, nullptr);
}

pf_status ensure_factor_storage(pf_ctx *ctx, int which, int prec) {
    Workspace &w = ctx->ws;
    const DevMat &m = ctx->dm[which];
    size_t sz = size_t(ctx->dc.ninst) * size_t(m.stride);
    if (!w.A[which]) TRY(dalloc(ctx, &w.A[which], sz));
    if (prec == PF_FP64 && !w.F64[which]) TRY(dalloc(ctx, &w.F64[which], sz));
    if (prec == PF_FP32 && !w.F32[which]) TRY(dalloc(ctx, &w.F32[which], sz));
    if (!w.fstatus[which][prec]) TRY(dalloc(ctx, &w.fstatus[which][prec], size_t(ctx->dc.ninst)));
    if (m.ft_ng > 0 && !w.TP[which][prec]) {
        const size_t np = size_t(ctx->dc.ninst) * size_t(m.ft_ng);
        if (prec == PF_FP64) TRY(dalloc(ctx, reinterpret_cast<double **>(&w.TP[which][prec]), np));
        else TRY(dalloc(ctx, reinterpret_cast<float **>(&w.TP[which][prec]), np));
    }
    if (m.npf3 > 0 && !w.TW[which][prec]) {
        if (prec == PF_FP64) TRY(dalloc(ctx, reinterpret_cast<double **>(&w.TW[which][prec]), size_t(m.tw_stride)));
        else TRY(dalloc(ctx, reinterpret_cast<float **>(&w.TW[which][prec]), size_t(m.tw_stride)));
    }
    if (m.npf3 > 0 && !w.TWd[which]) TRY(dalloc(ctx, &w.TWd[which], size_t(m.nt) * size_t(m.nt)));
    if (m.npf2 > 0 && !w.TV[which][prec]) {
        const size_t nt = size_t(ctx->dc.ninst) * size_t(m.tv_stride);
        if (prec == PF_FP64) TRY(dalloc(ctx, reinterpret_cast<double **>(&w.TV[which][prec]), nt));
        else TRY(dalloc(ctx, reinterpret_cast<float **>(&w.TV[which][prec]), nt));
    }
    if (!w.fdone[which]) {
        const size_t nd = size_t(ctx->dc.ninst) * size_t(std::max(1, m.n));
        TRY(dalloc(ctx, &w.fdone[which], nd));
        TRY(dalloc(ctx, &w.fsync[which], size_t(2)));
        TRY(dalloc(ctx, &w.famax[which], size_t(ctx->dc.ninst)));
        cudaError_t e = cudaMemset(w.fdone[which], 0, nd * sizeof(unsigned));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "factor flags");
        w.fepoch[which] = 0;
    }
    return PF_OK;
}

void free_case_storage(pf_ctx *ctx) {
    Workspace &w = ctx->ws;
    for (int a = 0; a < 2; a++) {
        dfree(ctx, w.A[a]); w.A[a] = nullptr;
        dfree(ctx, w.F64[a]); w.F64[a] = nullptr;
        dfree(ctx, w.F32[a]); w.F32[a] = nullptr;
        dfree(ctx, w.fdone[a]); w.fdone[a] = nullptr;
        dfree(ctx, w.LK[a]); w.LK[a] = nullptr;
        for (int b = 0; b < 2; b++) {
            dfree(ctx, w.LZ[a][b]); w.LZ[a][b] = nullptr;
            dfree(ctx, w.Lscr[a][b]); w.Lscr[a][b] = nullptr;
        }

        for (int b = 0; b < 2; b++) {
            dfree(ctx, w.TV[a][b]);
            w.TV[a][b] = nullptr;
            dfree(ctx, w.TP[a][b]);
            w.TP[a][b] = nullptr;
            dfree(ctx, w.TW[a][b]);
            w.TW[a][b] = nullptr;
        }
        dfree(ctx, w.TWd[a]);
        w.TWd[a] = nullptr;
        dfree(ctx, w.fsync[a]); w.fsync[a] = nullptr;
        dfree(ctx, w.famax[a]); w.famax[a] = nullptr;
        for (int b = 0; b < 2; b++) {
            dfree(ctx, w.fstatus[a][b]);
            w.fstatus[a][b] = nullptr;
            w.factored[a][b] = false;
        }
    }
    for (int q = 0; q < 2; q++) {
        dfree(ctx, w.JF[q]); w.JF[q] = nullptr;
        dfree(ctx, w.jfstat[q]); w.jfstat[q] = nullptr;
        w.jfactored[q] = false;
    }
    dfree(ctx, w.JA); w.JA = nullptr;
    {
        LaneSet &L = w.lanes;
        void *ptrs[] = {L.gcase, L.ginst, L.gshared, L.gown, L.owngroup, L.vm, L.va, L.cs, L.sn,
                        L.iv, L.e, L.f, L.psp, L.qsp, L.maxmis, L.lastmis, L.active, L.status,
                        L.iters, L.irs, L.nactive, L.X, L.b, L.x64, L.LF0, L.LF1};
        for (void *p : ptrs) dfree(ctx, p);
        L = LaneSet();
    }
    dfree(ctx, w.xg6); w.xg6 = nullptr;
    dfree(ctx, w.ef); w.ef = nullptr;
    dfree(ctx, w.vec); w.vec = nullptr;
    dfree(ctx, w.bmax); w.bmax = nullptr;
    dfree(ctx, w.iv); w.iv = nullptr;
    dfree(ctx, w.cstatus); w.cstatus = nullptr;
    dfree(ctx, w.res); w.res = nullptr;
    dfree(ctx, ctx->dc.outage); ctx->dc.outage = nullptr;
    dfree(ctx, ctx->dc.inst); ctx->dc.inst = nullptr;
    dfree(ctx, ctx->dc.inst_outage); ctx->dc.inst_outage = nullptr;
    dfree(ctx, ctx->dc.Psp); ctx->dc.Psp = nullptr;
    dfree(ctx, ctx->dc.Qsp); ctx->dc.Qsp = nullptr;
    dfree(ctx, w.lsbuf); w.lsbuf = nullptr;
    dfree(ctx, w.lsflag); w.lsflag = nullptr;
    w.case_out.clear();
    ctx->dc.ncase = 0;
    ctx->dc.ninst = 1;
}

pf_status assemble_ybus(pf_ctx *ctx, cudaStream_t s) {
    cudaError_t e = counted(ctx, PF_K_YBUS, 1, s, [&] { return launch_ybus(ctx->dn, s); });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ybus launch");
    return PF_OK;
}

// Assembles B' or B'' of the first ninst instances (-1: every instance)
// from the current admittance matrix.
pf_status assemble_matrix(pf_ctx *ctx, int which, int prec, cudaStream_t s, int ninst = -1) {
    TRY(ensure_factor_storage(ctx, which, prec));
    Workspace &w = ctx->ws;
    const DevMat &m = ctx->dm[which];
    cudaError_t e = counted(ctx, PF_K_ASSEMBLE, 1, s, [&] {
        return launch_assemble_slots(ctx->dn, ctx->dc, m, which, w.A[which], s, ninst);
    });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "assemble launch");
    return PF_OK;
}

// The next factorisation of matrix `which` (one instance) as a job of a
// packed factor launch: advances the matrix's flag epoch.
pf_status factor_job(pf_ctx *ctx, int which, int prec, FactorJob &J, cudaStream_t s) {
    Workspace &w = ctx->ws;
    const DevMat &m = ctx->dm[which];
    if (++w.fepoch[which] >= kGraphEpoch) {
        cudaError_t z = cudaMemsetAsync(w.fdone[which], 0,
                                        size_t(ctx->dc.ninst) * size_t(std::max(1, m.n)) * sizeof(unsigned), s);
        if (z != cudaSuccess) return cuda_fail(ctx, z, "factor flags");
        w.fepoch[which] = 1u;
    }
    J.m = m;
    J.A = w.A[which];
    J.F = prec == PF_FP64 ? (void *)w.F64[which] : (void *)w.F32[which];
    J.TV = w.TV[which][prec];
    J.fstatus = w.fstatus[which][prec];
    J.done = w.fdone[which];
    J.amax = w.famax[which];
    J.epoch = w.fepoch[which];
    return PF_OK;
}

// Assembles B' or B'' of every instance from the current admittance matrix
// and factorises them.
pf_status factor_matrix(pf_ctx *ctx, int which, int prec, cudaStream_t s, int blocks_per_sm = 2,
                        int ninst_f = -1) {
    const int nf = ninst_f > 0 ? ninst_f : ctx->dc.ninst;  // instances factorised (the first nf)
    // only those are assembled: with low-rank outages the outage instances'
    // matrices are the base one minus the branch's share (U S U^T), which
    // the iteration applies itself
    TRY(assemble_matrix(ctx, which, prec, s, nf));
    Workspace &w = ctx->ws;
    const DevMat &m = ctx->dm[which];
    cudaError_t e;
    void *F = prec == PF_FP64 ? (void *)w.F64[which] : (void *)w.F32[which];
    FactorSync fs;
    fs.done = w.fdone[which];
    fs.sync = w.fsync[which];
    fs.amax = w.famax[which];
    if (ctx->graph_capturing) {  // every replay clears the flags and publishes kGraphEpoch
        cudaError_t z = cudaMemsetAsync(w.fdone[which], 0,
                                        size_t(ctx->dc.ninst) * size_t(std::max(1, m.n)) * sizeof(unsigned), s);
        if (z != cudaSuccess) return cuda_fail(ctx, z, "factor flags");
        fs.epoch = kGraphEpoch;
    } else {
        if (++w.fepoch[which] >= kGraphEpoch) {  // wrapped: clear the flags, restart at 1
            cudaError_t z = cudaMemsetAsync(w.fdone[which], 0,
                                            size_t(ctx->dc.ninst) * size_t(std::max(1, m.n)) * sizeof(unsigned), s);
            if (z != cudaSuccess) return cuda_fail(ctx, z, "factor flags");
            w.fepoch[which] = 1u;
        }
        fs.epoch = w.fepoch[which];
    }
    fs.spin = 0;
    fs.nsm = ctx->num_sms;
    fs.mode = ctx->tune.factor;
    fs.blocks_per_sm = blocks_per_sm;
    fs.tail = ctx->tune.tail != 2;
    fs.smem_optin = ctx->smem_optin;
    fs.partg = w.TP[which][prec];
    // the tail factor of a few instances on a cluster of SMs each
    fs.tail_cluster = false;
    if (m.ft_ng > 0 && nf <= 8 && nf * kTailCtas <= ctx->num_sms) {
        int &cmax = ctx->tail_cl_max[which][prec];
        if (cmax < 0) cmax = factor_tail_clusters(m, prec);
        fs.tail_cluster = nf <= cmax;
    }
    e = counted(ctx, PF_K_FACTOR, 2, s, [&] {
        return launch_factor(m, prec, w.A[which], F, nf, w.fstatus[which][prec], fs, s);
    });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "factor launch");
    e = launch_tail_values(m, prec, F, w.TV[which][prec], nf, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tail values launch");
    if (ctx->tune.tail == 3 && m.npf3 > 0 && nf == 1) {
        e = counted(ctx, PF_K_FACTOR, 2, s, [&] {
            return launch_tail_w(m, prec, F, w.TWd[which], w.TW[which][prec], s);
        });
        if (e != cudaSuccess) return cuda_fail(ctx, e, "tail inverse launch");
    }
    w.factored[which][prec] = true;
    return PF_OK;
}

// Low-rank outages: Z and K of every outage instance of both matrices from
// the base factors (after factor_both with lowrank).
pf_status prepare_lowrank(pf_ctx *ctx, int prec, cudaStream_t s) {
    Workspace &w = ctx->ws;
    const int ninst = ctx->dc.ninst;
    const size_t elt = prec == PF_FP64 ? sizeof(double) : sizeof(float);
    for (int m = 0; m < 2; m++) {
        const DevMat &D = ctx->dm[m];
        if (!w.LZ[m][prec]) {
            const size_t nz = size_t(ninst) * 2 * size_t(std::max(1, D.n));
            const size_t ns = size_t(2 * (ninst - 1)) * size_t(std::max(1, D.n));
            if (prec == PF_FP64) {
                double *z = nullptr, *g = nullptr;
                TRY(dalloc(ctx, &z, nz));
                TRY(dalloc(ctx, &g, ns));
                w.LZ[m][prec] = z;
                w.Lscr[m][prec] = g;
            } else {
                float *z = nullptr, *g = nullptr;
                TRY(dalloc(ctx, &z, nz));
                TRY(dalloc(ctx, &g, ns));
                w.LZ[m][prec] = z;
                w.Lscr[m][prec] = g;
            }
            (void)elt;
        }
        if (!w.LK[m]) TRY(dalloc(ctx, &w.LK[m], size_t(8) * size_t(ninst)));
        const void *F = prec == PF_FP64 ? (const void *)w.F64[m] : (const void *)w.F32[m];
        const void *TV = ctx->tune.tail != 2 ? w.TV[m][prec] : nullptr;
        cudaError_t e = counted(ctx, PF_K_SOLVE, 2, s, [&] {
            return launch_lowrank(D, ctx->dn, ctx->dc, m, prec, F, TV, w.LZ[m][prec], w.LK[m],
                                  w.Lscr[m][prec], w.fstatus[m][prec], ctx->smem_optin, s);
        });
        if (e != cudaSuccess) return cuda_fail(ctx, e, "low-rank outages");
    }
    return PF_OK;
}

// B' and B'' of every instance.  With the dependency-driven factor (few
// instances) the two factorisations are independent chains of dependent
// columns: B'' runs on a second stream beside B', each launch capped at one
// block per SM so both are resident at once.
pf_status factor_both(pf_ctx *ctx, int prec, cudaStream_t s, bool lowrank, bool cl_inverse = false) {
    Workspace &w = ctx->ws;
    const int ninst = lowrank ? 1 : ctx->dc.ninst;
    const bool dep = ctx->tune.factor == 1 || (ctx->tune.factor == 0 && ninst < ctx->num_sms / 2);
    // the cluster engine's top inverse of a matrix follows that matrix's
    // factorisation on its own stream, so the shorter chain's inverse runs
    // while the longer chain is still factorising
    auto inverse = [&](int which, cudaStream_t st) -> pf_status {
        if (!cl_inverse) return PF_OK;
        cudaError_t e = counted(ctx, PF_K_FACTOR, 1, st, [&] {
            return launch_cl_inverse(ctx->cl[which], w.F64[which], ctx->clW[which], st);
        });
        return e == cudaSuccess ? PF_OK : cuda_fail(ctx, e, "top inverse");
    };
    if (!dep) {
        TRY(factor_matrix(ctx, PF_MAT_BP, prec, s, 2, ninst));
        TRY(inverse(PF_MAT_BP, s));
        TRY(factor_matrix(ctx, PF_MAT_BPP, prec, s, 2, ninst));
        TRY(inverse(PF_MAT_BPP, s));
        return PF_OK;
    }
    if (!w.side) {
        if (cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&w.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&w.join, cudaEventDisableTiming) != cudaSuccess)
            return fail(ctx, PF_ERR_CUDA, "side stream");
    }
    cudaError_t e = cudaEventRecord(w.fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(w.side, w.fork, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fork");
    TRY(factor_matrix(ctx, PF_MAT_BPP, prec, w.side, 1, ninst));
    TRY(inverse(PF_MAT_BPP, w.side));
    TRY(factor_matrix(ctx, PF_MAT_BP, prec, s, 1, ninst));
    TRY(inverse(PF_MAT_BP, s));
    e = cudaEventRecord(w.join, w.side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, w.join, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "join");
    return PF_OK;
}

// Lane groups of the current batch: shared-factor cases first, then
// own-factor (outage) cases, 32 lanes per group; state and vectors for prec.
pf_status ensure_lanes(pf_ctx *ctx, int prec) {
    LaneSet &L = ctx->ws.lanes;
    if (L.gcase && L.prec == prec) return PF_OK;
    if (L.gcase) {  // other precision: rebuild the precision-dependent arrays only
        dfree(ctx, L.X); dfree(ctx, L.LF0); dfree(ctx, L.LF1);
        L.X = L.LF0 = L.LF1 = nullptr;
    } else {
        const int ncase = ctx->dc.ncase;
        std::vector<int> inst(ncase);
        if (cudaMemcpy(inst.data(), ctx->dc.inst, sizeof(int) * ncase, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(ctx, PF_ERR_CUDA, "lanes: read instances");
        std::vector<int> sh, own;
        for (int c = 0; c < ncase; c++) (inst[c] == 0 ? sh : own).push_back(c);
        const int gs = (int(sh.size()) + 31) / 32, go = (int(own.size()) + 31) / 32;
        L.ngroups = gs + go;
        L.ncp = 32 * L.ngroups;
        L.nown = go;
        std::vector<int> gcase(L.ncp, -1), ginst(L.ncp, 0), gshared(L.ngroups), gown(L.ngroups, -1),
            owngroup(go);
        for (size_t q = 0; q < sh.size(); q++) gcase[q] = sh[q];
        for (size_t q = 0; q < own.size(); q++) {
            gcase[32 * gs + q] = own[q];
            ginst[32 * gs + q] = inst[own[q]];
        }
        for (int g = 0; g < L.ngroups; g++) {
            gshared[g] = g < gs ? 1 : 0;
            if (g >= gs) { gown[g] = g - gs; owngroup[g - gs] = g; }
        }
        TRY(upload(ctx, &L.gcase, gcase.data(), gcase.size()));
        TRY(upload(ctx, &L.ginst, ginst.data(), ginst.size()));
        TRY(upload(ctx, &L.gshared, gshared.data(), gshared.size()));
        TRY(upload(ctx, &L.gown, gown.data(), gown.size()));
        TRY(upload(ctx, &L.owngroup, owngroup.data(), std::max<size_t>(1, owngroup.size())));
        const size_t ns = size_t(ctx->nbus) * L.ncp;
        double **st[] = {&L.vm, &L.va, &L.cs, &L.sn, &L.iv, &L.e, &L.f, &L.psp, &L.qsp};
        for (double **p : st) TRY(dalloc(ctx, p, ns));
        TRY(dalloc(ctx, &L.maxmis, size_t(L.ncp)));
        TRY(dalloc(ctx, &L.lastmis, size_t(L.ncp)));
        TRY(dalloc(ctx, &L.active, size_t(L.ncp)));
        TRY(dalloc(ctx, &L.status, size_t(L.ncp)));
        TRY(dalloc(ctx, &L.iters, size_t(L.ncp)));
        TRY(dalloc(ctx, &L.irs, size_t(L.ncp)));
        TRY(dalloc(ctx, &L.nactive, size_t(1)));
        TRY(dalloc(ctx, &L.b, ns));
        TRY(dalloc(ctx, &L.x64, ns));
        if (cudaMemset(L.maxmis, 0, sizeof(double) * L.ncp) != cudaSuccess)
            return fail(ctx, PF_ERR_CUDA, "memset");
    }
    const size_t ns = size_t(ctx->nbus) * L.ncp;
    const size_t nl0 = size_t(std::max(1, L.nown)) * ctx->dm[0].stride * 32;
    const size_t nl1 = size_t(std::max(1, L.nown)) * ctx->dm[1].stride * 32;
    if (prec == PF_FP64) {
        double *x = nullptr, *l0 = nullptr, *l1 = nullptr;
        TRY(dalloc(ctx, &x, ns)); TRY(dalloc(ctx, &l0, nl0)); TRY(dalloc(ctx, &l1, nl1));
        L.X = x; L.LF0 = l0; L.LF1 = l1;
    } else {
        float *x = nullptr, *l0 = nullptr, *l1 = nullptr;
        TRY(dalloc(ctx, &x, ns)); TRY(dalloc(ctx, &l0, nl0)); TRY(dalloc(ctx, &l1, nl1));
        L.X = x; L.LF0 = l0; L.LF1 = l1;
    }
    L.prec = prec;
    return PF_OK;
}

pf_status ensure_nr_storage(pf_ctx *ctx, int prec) {
    Workspace &w = ctx->ws;
    const DevMat &m = ctx->dm[PF_MAT_BP];
    const size_t n = size_t(ctx->dc.ncase) * size_t(m.jstride);
    if (!w.JA) TRY(dalloc(ctx, &w.JA, n));
    if (!w.xg6) TRY(dalloc(ctx, &w.xg6, size_t(ctx->dc.ncase) * 6 * ctx->nbus));
    if (!w.JF[prec]) {
        if (prec == PF_FP64) {
            double *p = nullptr;
            TRY(dalloc(ctx, &p, n));
            w.JF[prec] = p;
        } else {
            float *p = nullptr;
            TRY(dalloc(ctx, &p, n));
            w.JF[prec] = p;
        }
    }
    if (!w.jfstat[prec]) TRY(dalloc(ctx, &w.jfstat[prec], size_t(ctx->dc.ncase)));
    if (!w.jdone) {
        const size_t nd = size_t(ctx->dc.ncase) * size_t(std::max(1, m.n));
        TRY(dalloc(ctx, &w.jdone, nd));
        TRY(dalloc(ctx, &w.jsync, size_t(2) * size_t(ctx->dc.ncase)));
        cudaError_t e = cudaMemset(w.jdone, 0, nd * sizeof(unsigned));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "jacobian flags");
        w.jepoch = 0;
    }
    return PF_OK;
}

NrLaunch nr_launch(pf_ctx *ctx, int prec) {
    Workspace &w = ctx->ws;
    NrLaunch L;
    L.dn = ctx->dn;
    L.dc = ctx->dc;
    L.m = ctx->dm[PF_MAT_BP];
    L.F = w.JF[prec];
    L.A = w.JA;
    L.fstat = w.jfstat[prec];
    L.prec = prec;
    L.ef = w.ef;
    L.xg = w.xg6;
    L.bmax = w.bmax;
    L.res = w.res;
    L.smem_optin = ctx->smem_optin;
    L.cluster = nr_cluster_size(L.m, ctx->dc.ncase, ctx->num_sms, prec, ctx->smem_optin);
    L.jdone = w.jdone;
    L.jsync = w.jsync;
    return L;
}

// Whether a run can use the cluster engine: FDPF in FP64 on one case of the
// base network (no outage instance), with both programs fitting one CTA's
// shared memory and a 16-block cluster resident.
bool cluster_applies(pf_ctx *ctx, const pf_run_opts *o) {
    if (o->method != PF_FDPF || o->precision != PF_FP64 || ctx->dc.ncase != 1 || ctx->dc.ninst != 1)
        return false;
    if (!ctx->hcl[0].ok || !ctx->hcl[1].ok) return false;
    if (ctx->cl_smem + 4096 > ctx->smem_optin || ctx->num_sms < kClCtas) return false;
    return fdpf_cl_fits(ctx->cl_smem);
}

pf_status ensure_cluster(pf_ctx *ctx) {
    if (ctx->cl[0].tasks) return PF_OK;
    for (int w = 0; w < 2; w++) TRY(upload_cluster(ctx, w));
    return PF_OK;
}

// Rebuilds the cluster engine's programs with g subtree levels per step:
// the device copies are freed (uploaded again on the next use) and a CUDA
// graph that launched the old ones is dropped.
pf_status set_cluster_group(pf_ctx *ctx, int g) {
    if (g == ctx->cl_group) return PF_OK;
    drop_graph(ctx);
    for (int w = 0; w < 2; w++) {
        ClMat &M = ctx->cl[w];
        void *ptrs[] = {M.tpar, M.tcp, M.tcdep, M.tcpos, M.tdepth, M.vsrc, M.vals, M.tasks, M.tptr, M.steps,
                        M.sptr, M.refs, M.eptr, M.vptr, M.rhsref, M.xref, M.gw_col, M.gw_upd, M.gm_ptr,
                        M.gm_term, M.gv};
        for (void *p : ptrs) dfree(ctx, p);
        dfree(ctx, ctx->clW[w]);
        ctx->clW[w] = nullptr;
        M = ClMat();
    }
    ctx->cl_group = g;
    for (int w = 0; w < 2; w++) TRY(build_cluster(ctx, w, ctx->hcl[w], g));
    ctx->cl_smem = cluster_smem_layout(ctx);
    return PF_OK;
}

// Epochs for the Jacobian factorisations of one NR or adjoint launch (at
// most `count`); the flags are cleared when the counter would wrap.
unsigned nr_epochs(pf_ctx *ctx, unsigned count, cudaStream_t s) {
    Workspace &w = ctx->ws;
    if (w.jepoch > 0xF0000000u) {
        cudaMemsetAsync(w.jdone, 0, size_t(ctx->dc.ncase) * size_t(std::max(1, ctx->dm[0].n)) * sizeof(unsigned), s);
        w.jepoch = 0;
    }
    const unsigned e0 = w.jepoch;
    w.jepoch += count;
    return e0;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

pf_status pf_create(const pf_bus *bus, int32_t nbus, const pf_branch *branch, int32_t nbranch,
                    pf_ctx **out) {
    if (!out) return PF_ERR_ARG;
    *out = nullptr;
    if (!bus || nbus < 2 || nbranch < 1 || !branch) return PF_ERR_ARG;
    pf_ctx *ctx = new (std::nothrow) pf_ctx();
    if (!ctx) return PF_ERR_OOM;
    auto reject = [&](pf_status st) {
        // keep the context alive only long enough to report
        delete ctx;
        return st;
    };
    ctx->nbus = nbus;
    ctx->nbr = nbranch;
    ctx->bus.assign(bus, bus + nbus);
    ctx->branch.assign(branch, branch + nbranch);
    int nslack = 0;
    for (int i = 0; i < nbus; i++) {
        const pf_bus &b = bus[i];
        if (b.type < PF_BUS_PQ || b.type > PF_BUS_SLACK) return reject(PF_ERR_ARG);
        if (b.type == PF_BUS_SLACK) { nslack++; ctx->slack = i; }
        double v[7] = {b.pd, b.qd, b.gs, b.bs, b.pg, b.vset, b.va};
        for (double x : v)
            if (!std::isfinite(x)) return reject(PF_ERR_ARG);
        if (b.type != PF_BUS_PQ && !(b.vset > 0)) return reject(PF_ERR_ARG);
    }
    if (nslack != 1) return reject(PF_ERR_ARG);
    std::vector<std::vector<int>> adj(nbus);
    for (int e = 0; e < nbranch; e++) {
        const pf_branch &r = branch[e];
        if (r.from < 0 || r.from >= nbus || r.to < 0 || r.to >= nbus || r.from == r.to)
            return reject(PF_ERR_ARG);
        double v[4] = {r.r, r.x, r.b, r.tap};
        for (double x : v)
            if (!std::isfinite(x)) return reject(PF_ERR_ARG);
        if (r.x == 0.0 || r.tap < 0.0) return reject(PF_ERR_ARG);
        if (r.status != 0 && r.status != 1) return reject(PF_ERR_ARG);
        adj[r.from].push_back(r.to);
        adj[r.to].push_back(r.from);
    }
    // connectivity to the slack through in-service branches
    {
        std::vector<std::vector<int>> live(nbus);
        for (int e = 0; e < nbranch; e++)
            if (branch[e].status) {
                live[branch[e].from].push_back(branch[e].to);
                live[branch[e].to].push_back(branch[e].from);
            }
        std::vector<char> seen(nbus, 0);
        std::vector<int> stack{ctx->slack};
        seen[ctx->slack] = 1;
        int cnt = 1;
        while (!stack.empty()) {
            int v = stack.back();
            stack.pop_back();
            for (int u : live[v])
                if (!seen[u]) { seen[u] = 1; cnt++; stack.push_back(u); }
        }
        if (cnt != nbus) return reject(PF_ERR_ISLAND);
    }
    // Ybus pattern: diagonal plus one entry per adjacent bus, ascending
    ctx->rowptr.assign(nbus + 1, 0);
    for (int i = 0; i < nbus; i++) {
        adj[i].push_back(i);
        std::sort(adj[i].begin(), adj[i].end());
        adj[i].erase(std::unique(adj[i].begin(), adj[i].end()), adj[i].end());
        ctx->rowptr[i + 1] = ctx->rowptr[i] + int(adj[i].size());
    }
    ctx->col.reserve(ctx->rowptr[nbus]);
    for (int i = 0; i < nbus; i++) ctx->col.insert(ctx->col.end(), adj[i].begin(), adj[i].end());

    // host index tables used by the device kernels
    ctx->ydiag.assign(nbus, 0);
    ctx->inc_ptr.assign(nbus + 1, 0);
    ctx->inc_br.assign(2 * size_t(nbranch), 0);
    ctx->inc_side.assign(2 * size_t(nbranch), 0);
    ctx->inc_pos.assign(2 * size_t(nbranch), 0);
    ctx->br_pos.assign(4 * size_t(nbranch), 0);
    for (int i = 0; i < nbus; i++) ctx->ydiag[i] = ypos(ctx, i, i);
    for (int e = 0; e < nbranch; e++) { ctx->inc_ptr[branch[e].from + 1]++; ctx->inc_ptr[branch[e].to + 1]++; }
    for (int i = 0; i < nbus; i++) ctx->inc_ptr[i + 1] += ctx->inc_ptr[i];
    {
        std::vector<int> f(ctx->inc_ptr.begin(), ctx->inc_ptr.end() - 1);
        for (int e = 0; e < nbranch; e++) {  // ascending branch index per bus
            const int a = branch[e].from, b = branch[e].to;
            int q = f[a]++;
            ctx->inc_br[q] = e; ctx->inc_side[q] = 0; ctx->inc_pos[q] = ypos(ctx, a, b);
            q = f[b]++;
            ctx->inc_br[q] = e; ctx->inc_side[q] = 1; ctx->inc_pos[q] = ypos(ctx, b, a);
        }
    }
    {   // per off-diagonal entry, in row order, the branches reaching it in
        // the order of its row's incidence list (ascending branch index)
        std::vector<std::vector<int>> at(ctx->col.size());
        for (int i = 0; i < nbus; i++)
            for (int q = ctx->inc_ptr[i]; q < ctx->inc_ptr[i + 1]; q++) at[ctx->inc_pos[q]].push_back(ctx->inc_br[q]);
        ctx->yoff.clear();
        ctx->yoff_br.clear();
        for (int i = 0; i < nbus; i++)
            for (int p = ctx->rowptr[i]; p < ctx->rowptr[i + 1]; p++) {
                if (p == ctx->ydiag[i]) continue;
                const int lo = int(ctx->yoff_br.size());
                ctx->yoff_br.insert(ctx->yoff_br.end(), at[p].begin(), at[p].end());
                ctx->yoff.push_back(int4{p, lo, int(ctx->yoff_br.size()), 0});
            }
    }
    {   // the mismatch's thread order: buses by row length within a range
        auto by_len = [&](std::vector<int> &ord, int i0, int i1) {
            std::stable_sort(ord.begin() + i0, ord.begin() + i1, [&](int x, int y) {
                return ctx->rowptr[x + 1] - ctx->rowptr[x] < ctx->rowptr[y + 1] - ctx->rowptr[y];
            });
        };
        ctx->mis_ord.resize(nbus);
        for (int i = 0; i < nbus; i++) ctx->mis_ord[i] = i;
        ctx->mis_ord_cl = ctx->mis_ord;
        // within windows of 1,024 consecutive buses: a warp's rows of one
        // length while the block's accesses stay within a window's sectors
        for (int i0 = 0; i0 < nbus; i0 += 1024) by_len(ctx->mis_ord, i0, std::min(nbus, i0 + 1024));
        const int slice = (nbus + kClCtas - 1) / kClCtas;  // the cluster engine's bus slices
        for (int r = 0; r < kClCtas; r++) {
            const int i0 = std::min(nbus, r * slice), i1 = std::min(nbus, i0 + slice);
            by_len(ctx->mis_ord_cl, i0, i1);
        }
    }
    for (int e = 0; e < nbranch; e++) {
        const int a = branch[e].from, b = branch[e].to;
        ctx->br_pos[4 * e + 0] = ctx->ydiag[a];
        ctx->br_pos[4 * e + 1] = ctx->ydiag[b];
        ctx->br_pos[4 * e + 2] = ypos(ctx, a, b);
        ctx->br_pos[4 * e + 3] = ypos(ctx, b, a);
    }
    *out = ctx;
    return PF_OK;
}

pf_status pf_analyze(pf_ctx *ctx, pf_symbolic_info *info) {
    if (!ctx) return PF_ERR_ARG;
    auto t0 = std::chrono::steady_clock::now();
    if (!ctx->analyzed) {
        for (int w = 0; w < 2; w++) {
            TRY(analyze_matrix(ctx, w, ctx->hm[w]));
            if (ctx->on_device) TRY(upload_matrix(ctx, ctx->hm[w], ctx->dm[w]));
        }
        for (int w = 0; w < 2; w++) TRY(build_cluster(ctx, w, ctx->hcl[w], ctx->cl_group));
        ctx->cl_smem = cluster_smem_layout(ctx);
        ctx->analyzed = true;
    }
    auto t1 = std::chrono::steady_clock::now();
    if (info) {
        memset(info, 0, sizeof(*info));
        for (int w = 0; w < 2; w++) {
            info->n[w] = ctx->hm[w].n;
            info->nnz_l[w] = ctx->hm[w].Lp[ctx->hm[w].n];
            info->nlevels[w] = ctx->hm[w].nlev;
            info->max_col[w] = ctx->hm[w].max_col;
            info->nupdates[w] = ctx->hm[w].nupd;
        }
        info->nnz_ybus = ctx->rowptr[ctx->nbus];
        info->analyze_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    }
    return PF_OK;
}

pf_status pf_get_symbolic(const pf_ctx *ctx, int32_t which, int32_t *perm, int32_t *parent,
                          int32_t *level, int64_t *Lp, int32_t *Li) {
    if (!ctx || (which != PF_MAT_BP && which != PF_MAT_BPP)) return PF_ERR_ARG;
    if (!ctx->analyzed) return PF_ERR_STATE;
    const HostMat &H = ctx->hm[which];
    if (perm) std::copy(H.perm.begin(), H.perm.end(), perm);
    if (parent) std::copy(H.parent.begin(), H.parent.end(), parent);
    if (level) std::copy(H.level.begin(), H.level.end(), level);
    if (Lp) std::copy(H.Lp.begin(), H.Lp.end(), Lp);
    if (Li) std::copy(H.Li.begin(), H.Li.end(), Li);
    return PF_OK;
}

pf_status pf_set_cases(pf_ctx *ctx, int32_t ncase, const double *load_scale,
                       const int32_t *outage) {
    if (!ctx || ncase < 1) return fail(ctx, PF_ERR_ARG, "ncase must be >= 1");
    if (!ctx->analyzed) return fail(ctx, PF_ERR_STATE, "pf_analyze first");
    std::vector<int> out(ncase, -1), inst(ncase, 0), inst_out(1, -1);
    for (int c = 0; c < ncase; c++) {
        if (outage) {
            if (outage[c] < -1 || outage[c] >= ctx->nbr)
                return fail(ctx, PF_ERR_ARG, "outage[%d] = %d out of range", c, outage[c]);
            out[c] = outage[c];
        }
        if (out[c] >= 0) {
            inst[c] = int(inst_out.size());
            inst_out.push_back(out[c]);
        }
    }
    const size_t nls = size_t(ncase) * size_t(ctx->nbus);
    Workspace &w0 = ctx->ws;
    if (ctx->on_device && ctx->dc.ncase == ncase && w0.ncase_alloc == ncase && w0.lsbuf && w0.lsflag &&
        w0.case_out == out) {
        // the same cases with new loads: the batch's arrays, factors and CUDA
        // graph stay; only the specified injections are formed again.  Many
        // scales (a batch's) are checked on the device instead of by a host
        // loop: non-finite ones leave the injections unchanged.
        const bool dev_check = load_scale && nls > (size_t(1) << 20);
        if (load_scale && !dev_check)
            for (size_t q = 0; q < nls; q++)
                if (!std::isfinite(load_scale[q])) return fail(ctx, PF_ERR_ARG, "non-finite load scale");
        cudaError_t e = cudaSuccess;
        int bad = 0;
        if (dev_check) e = cudaMemsetAsync(w0.lsflag, 0, sizeof(int), 0);
        if (e == cudaSuccess && load_scale)
            e = cudaMemcpyAsync(w0.lsbuf, load_scale, sizeof(double) * nls, cudaMemcpyHostToDevice, 0);
        if (e == cudaSuccess && dev_check) e = launch_finite_check(w0.lsbuf, (long long)nls, w0.lsflag, 0);
        if (e == cudaSuccess)
            e = counted(ctx, PF_K_SPEC, 1, 0, [&] {
                return launch_case_spec(ctx->dn, ctx->dc, load_scale ? w0.lsbuf : nullptr, 0,
                                        dev_check ? w0.lsflag : nullptr);
            });
        if (e == cudaSuccess && dev_check) e = cudaMemcpyAsync(&bad, w0.lsflag, sizeof(int), cudaMemcpyDeviceToHost, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "case spec");
        if (bad) return fail(ctx, PF_ERR_ARG, "non-finite load scale");
        return PF_OK;
    }
    if (load_scale)
        for (size_t q = 0; q < nls; q++)
            if (!std::isfinite(load_scale[q])) return fail(ctx, PF_ERR_ARG, "non-finite load scale");
    TRY(ensure_device(ctx));
    drop_graph(ctx);  // its launches point into the batch's arrays
    ctx->set_gen++;
    free_case_storage(ctx);
    DevCases &dc = ctx->dc;
    dc.ncase = ncase;
    dc.ninst = int(inst_out.size());
    TRY(upload(ctx, &dc.outage, out.data(), out.size()));
    TRY(upload(ctx, &dc.inst, inst.data(), inst.size()));
    TRY(upload(ctx, &dc.inst_outage, inst_out.data(), inst_out.size()));
    TRY(dalloc(ctx, &dc.Psp, size_t(ncase) * ctx->nbus));
    TRY(dalloc(ctx, &dc.Qsp, size_t(ncase) * ctx->nbus));
    Workspace &w = ctx->ws;
    TRY(dalloc(ctx, &w.lsbuf, size_t(ncase) * ctx->nbus));
    TRY(dalloc(ctx, &w.lsflag, 1));
    cudaError_t e = cudaSuccess;
    if (load_scale)
        e = cudaMemcpy(w.lsbuf, load_scale, sizeof(double) * size_t(ncase) * ctx->nbus, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = counted(ctx, PF_K_SPEC, 1, 0, [&] { return launch_case_spec(ctx->dn, dc, load_scale ? w.lsbuf : nullptr, 0); });
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "case spec");
    w.case_out = out;
    TRY(dalloc(ctx, &w.ef, size_t(ncase) * 4 * ctx->nbus));
    TRY(dalloc(ctx, &w.vec, size_t(ncase) * 3 * ctx->nbus));
    TRY(dalloc(ctx, &w.bmax, size_t(ncase) * 16));
    TRY(dalloc(ctx, &w.iv, size_t(ncase) * ctx->nbus));
    TRY(dalloc(ctx, &w.cstatus, size_t(ncase)));
    if (cudaMemset(w.cstatus, 0, sizeof(int) * ncase) != cudaSuccess)
        return fail(ctx, PF_ERR_CUDA, "memset");
    TRY(dalloc(ctx, &w.res, size_t(ncase)));
    w.ncase_alloc = ncase;
    return PF_OK;
}

pf_status pf_set_injections(pf_ctx *ctx, const double *psp_dev, const double *qsp_dev,
                            void *stream) {
    if (!ctx || !psp_dev || !qsp_dev) return fail(ctx, PF_ERR_ARG, "null pointer");
    if (!ctx->analyzed) return fail(ctx, PF_ERR_STATE, "pf_analyze first");
    TRY(ensure_cases(ctx));
    const size_t bytes = sizeof(double) * size_t(ctx->dc.ncase) * ctx->nbus;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(ctx->dc.Psp, psp_dev, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->dc.Qsp, qsp_dev, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set injections");
    return PF_OK;
}

pf_status pf_factor(pf_ctx *ctx, int32_t which, int32_t precision, void *stream) {
    if (!ctx || (which != PF_MAT_BP && which != PF_MAT_BPP) ||
        (precision != PF_FP64 && precision != PF_FP32))
        return fail(ctx, PF_ERR_ARG, "bad matrix or precision");
    if (!ctx->analyzed) return fail(ctx, PF_ERR_STATE, "pf_analyze first");
    TRY(ensure_cases(ctx));
    TRY(assemble_ybus(ctx, (cudaStream_t)stream));
    return factor_matrix(ctx, which, precision, (cudaStream_t)stream);
}

pf_status pf_get_factor(pf_ctx *ctx, int32_t which, int32_t precision, int32_t c, double *D,
                        double *Lx, int32_t *status) {
    if (!ctx || (which != PF_MAT_BP && which != PF_MAT_BPP) ||
        (precision != PF_FP64 && precision != PF_FP32))
        return fail(ctx, PF_ERR_ARG, "bad matrix or precision");
    if (!ctx->ws.factored[which][precision]) return fail(ctx, PF_ERR_STATE, "not factored");
    if (c < 0 || c >= ctx->dc.ncase) return fail(ctx, PF_ERR_ARG, "case out of range");
    const DevMat &m = ctx->dm[which];
    const HostMat &H = ctx->hm[which];
    int inst = 0;
    cudaError_t e = cudaMemcpy(&inst, ctx->dc.inst + c, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "get_factor");
    std::vector<double> v(m.offLc + m.nnz);
    if (precision == PF_FP64) {
        e = cudaMemcpy(v.data(), ctx->ws.F64[which] + size_t(inst) * m.stride,
                       sizeof(double) * v.size(), cudaMemcpyDeviceToHost);
    } else {
        std::vector<float> f(v.size());
        e = cudaMemcpy(f.data(), ctx->ws.F32[which] + size_t(inst) * m.stride,
                       sizeof(float) * f.size(), cudaMemcpyDeviceToHost);
        for (size_t q = 0; q < f.size(); q++) v[q] = f[q];
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "get_factor");
    // back to step numbering
    if (D)
        for (int st = 0; st < m.n; st++) D[st] = v[H.new_of_step[st]];
    if (Lx)
        for (int p = 0; p < m.nnz; p++) Lx[p] = v[m.offLc + H.csc_of_steppos[p]];
    if (status) {
        e = cudaMemcpy(status, ctx->ws.fstatus[which][precision] + inst, sizeof(int),
                       cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "get_factor status");
    }
    return PF_OK;
}

pf_status pf_solve(pf_ctx *ctx, int32_t which, int32_t precision, int32_t transpose,
                   double *rhs_inout_dev, int32_t ncase, void *stream) {
    (void)transpose;  // B' and B'' are symmetric
    if (!ctx || (which != PF_MAT_BP && which != PF_MAT_BPP) || !rhs_inout_dev ||
        (precision != PF_FP64 && precision != PF_FP32))
        return fail(ctx, PF_ERR_ARG, "bad argument");
    if (!ctx->ws.factored[which][precision]) return fail(ctx, PF_ERR_STATE, "pf_factor first");
    if (ncase < 1 || ncase > ctx->dc.ncase) return fail(ctx, PF_ERR_ARG, "ncase out of range");
    const void *F = precision == PF_FP64 ? (const void *)ctx->ws.F64[which]
                                         : (const void *)ctx->ws.F32[which];
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = counted(ctx, PF_K_SOLVE, 1, s, [&] {
        return launch_solve(ctx->dm[which], precision, F,
                            ctx->tune.tail != 2 ? ctx->ws.TV[which][precision] : nullptr, ctx->dc.inst,
                            rhs_inout_dev, ncase, ctx->ws.vec, ctx->ws.cstatus, ctx->smem_optin, s);
    });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "solve launch");
    return PF_OK;
}

pf_status pf_mismatch(pf_ctx *ctx, const double *vm_dev, const double *va_dev, double *dp_dev,
                      double *dq_dev, double *maxmis_dev, int32_t ncase, void *stream) {
    if (!ctx || !vm_dev || !va_dev || !dp_dev || !dq_dev || !maxmis_dev)
        return fail(ctx, PF_ERR_ARG, "null pointer");
    if (!ctx->analyzed) return fail(ctx, PF_ERR_STATE, "pf_analyze first");
    TRY(ensure_cases(ctx));
    if (ncase < 1 || ncase > ctx->dc.ncase) return fail(ctx, PF_ERR_ARG, "ncase out of range");
    cudaStream_t s = (cudaStream_t)stream;
    TRY(assemble_ybus(ctx, s));
    cudaError_t e = counted(ctx, PF_K_MISMATCH, 2, s, [&] {
        return launch_mismatch(ctx->dn, ctx->dc, vm_dev, va_dev, dp_dev, dq_dev, maxmis_dev,
                               ctx->ws.ef, ncase, s);
    });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mismatch launch");
    return PF_OK;
}

}  // extern "C"

namespace {
pf_status run_once(pf_ctx *ctx, const pf_run_opts *opts, double *vm_dev, double *va_dev,
                   pf_case_result *res_host, void *stream);
}  // namespace

extern "C" {

pf_status pf_run_to_tol(pf_ctx *ctx, const pf_run_opts *opts, double *vm_dev, double *va_dev,
                        pf_case_result *res_host, void *stream) {
    return run_once(ctx, opts, vm_dev, va_dev, res_host, stream);
}

}  // extern "C"

namespace {
// Device work of one fast decoupled run on the block or the cluster engine,
// enqueued on s without any host synchronisation: the admittance matrix,
// B' and B'' assembled and factorised (B'' on the side stream), then the
// low-rank outage data or the tail inverses, then the iteration kernel.
pf_status issue_fdpf(pf_ctx *ctx, const pf_run_opts *opts, double *vm_dev, double *va_dev, int engine,
                     cudaStream_t s) {
    Workspace &w = ctx->ws;
    const int prec = opts->precision;
    TRY(assemble_ybus(ctx, s));
    // FDPF -> NR fallback (Section III): unconverged cases switch to
    // Newton-Raphson from a flat start inside the iteration launch
    NrLaunch fbl;
    const NrLaunch *fb = nullptr;
    if (opts->fallback) {
        TRY(ensure_nr_storage(ctx, prec));
        fbl = nr_launch(ctx, prec);
        fbl.o = *opts;
        fbl.o.method = PF_NR;
        fbl.o.max_iter = kFallbackIters;
        fbl.o.flat_start = 1;
        fbl.vm = vm_dev;
        fbl.va = va_dev;
        if (ctx->graph_capturing) {  // every replay clears the flags and counts from kNrGraphEpoch
            cudaError_t e = cudaMemsetAsync(
                w.jdone, 0, size_t(ctx->dc.ncase) * size_t(std::max(1, ctx->dm[0].n)) * sizeof(unsigned), s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "fallback flags");
            fbl.epoch0 = kNrGraphEpoch;
        } else {
            fbl.epoch0 = nr_epochs(ctx, unsigned(kFallbackIters) + 2u, s);
        }
        fb = &fbl;
    }
    if (engine == PF_ENGINE_CLUSTER) {
        TRY(ensure_cluster(ctx));
        TRY(factor_both(ctx, prec, s, false, true));
        cudaError_t e = counted(ctx, PF_K_FACTOR, 1, s, [&] {
            return launch_cl_prepare(ctx->cl[0], ctx->cl[1], w.F64[0], w.F64[1], ctx->clW[0], ctx->clW[1], s);
        });
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cluster prepare");
        e = counted(ctx, PF_K_RUN, 1, s, [&] {
            return launch_fdpf_cl(ctx->dn, ctx->dc, ctx->cl[0], ctx->cl[1], w.fstatus[0][prec],
                                  w.fstatus[1][prec], *opts, vm_dev, va_dev, w.ef, w.iv, w.bmax, w.res,
                                  ctx->cl_smem, s, fb, ctx->smem_optin);
        });
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cluster fdpf launch");
        return PF_OK;
    }
    const bool lowrank = ctx->tune.outage == 2 && ctx->dc.ninst > 1;
    TRY(factor_both(ctx, prec, s, lowrank));
    if (lowrank) {
        TRY(prepare_lowrank(ctx, prec, s));
        // the outage instances' own factors were not computed: pf_solve and
        // pf_get_factor need pf_factor first
        w.factored[0][prec] = w.factored[1][prec] = false;
    }
    const void *F0 = prec == PF_FP64 ? (const void *)w.F64[0] : (const void *)w.F32[0];
    const void *F1 = prec == PF_FP64 ? (const void *)w.F64[1] : (const void *)w.F32[1];
    int cl = fdpf_cluster_size(ctx->dc.ncase, ctx->num_sms, prec, ctx->smem_optin,
                               std::max(ctx->dm[0].n, ctx->dm[1].n));
    if (ctx->tune.cluster > 0 && ctx->tune.cluster < cl) cl = ctx->tune.cluster < 8 ? 1 : 8;
    const bool tail = ctx->tune.tail != 2;
    // tail form 3: every case's solves use the factor of instance 0
    const bool tw = ctx->tune.tail == 3 && (ctx->dc.ninst == 1 || lowrank);
    cudaError_t e = counted(ctx, PF_K_RUN, 1, s, [&] {
        return launch_fdpf(ctx->dn, ctx->dc, ctx->dm, prec, F0, F1, tail ? w.TV[0][prec] : nullptr,
                           tail ? w.TV[1][prec] : nullptr, w.A[0], w.A[1], w.fstatus[0][prec],
                           w.fstatus[1][prec], *opts, vm_dev, va_dev, w.ef, w.iv, w.vec, w.bmax, w.res,
                           ctx->smem_optin, ctx->smem_per_sm, cl, ctx->tune.threads, s,
                           lowrank ? w.LZ[0][prec] : nullptr,
                           lowrank ? w.LZ[1][prec] : nullptr, lowrank ? w.LK[0] : nullptr,
                           lowrank ? w.LK[1] : nullptr, fb, tw ? w.TW[0][prec] : nullptr,
                           tw ? w.TW[1][prec] : nullptr);
    });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fdpf launch");
    return PF_OK;
}


// The device work of a run, from a CUDA graph when the same arguments come
// again: the first call with a set of arguments runs directly (allocating
// whatever it needs), the second captures the work on the context's own
// stream, instantiates it and launches it on s, later ones only launch it.
// The key is everything the captured launches bake in: the state pointers,
// the options, the tuning, the engine and the batch (set_gen changes with
// every pf_set_cases and pf_set_injections keeps the arrays in place).
// With profiling on, or after a capture that failed, runs are direct.
pf_status run_device_work(pf_ctx *ctx, const pf_run_opts *opts, double *vm_dev, double *va_dev, int engine,
                          cudaStream_t s) {
    std::vector<unsigned char> key(2 * sizeof(void *) + sizeof(pf_run_opts) + 6 * sizeof(int32_t) +
                                   3 * sizeof(int));
    unsigned char *k = key.data();
    auto put = [&](const void *p, size_t n) {
        memcpy(k, p, n);
        k += n;
    };
    put(&vm_dev, sizeof(void *));
    put(&va_dev, sizeof(void *));
    pf_run_opts o;
    memset(&o, 0, sizeof(o));
    o.method = opts->method;
    o.precision = opts->precision;
    o.tol = opts->tol;
    o.max_iter = opts->max_iter;
    o.ir_max = opts->ir_max;
    o.ir_tol = opts->ir_tol;
    o.ir_abs = opts->ir_abs;
    o.flat_start = opts->flat_start;
    o.spin_limit = opts->spin_limit;
    o.engine = opts->engine;
    o.fallback = opts->fallback;
    put(&o, sizeof(o));
    const int32_t t[6] = {ctx->tune.engine, ctx->tune.cluster, ctx->tune.factor, ctx->tune.tail,
                          ctx->tune.outage, ctx->tune.threads};
    put(t, sizeof(t));
    const int extra[3] = {engine, ctx->set_gen, ctx->dc.ncase};
    put(extra, sizeof(extra));
    const bool graphs = !ctx->profiling && !ctx->graphs_off;
    if (graphs && ctx->gexec && key == ctx->gkey) {
        cudaError_t e = cudaGraphLaunch(ctx->gexec, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
        for (int q = 0; q < PF_K_COUNT; q++) ctx->kstat[q].launches += ctx->glaunches[q];
        return PF_OK;
    }
    if (!graphs || key != ctx->gkey_last) {
        ctx->gkey_last = key;
        return issue_fdpf(ctx, opts, vm_dev, va_dev, engine, s);
    }
    // the same arguments a second time: capture
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
    ctx->gkey.clear();
    if (!ctx->gstream && cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ctx->graphs_off = true;
        return issue_fdpf(ctx, opts, vm_dev, va_dev, engine, s);
    }
    for (int q = 0; q < PF_K_COUNT; q++) ctx->glaunches[q] = 0;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeRelaxed);
    pf_status st = PF_ERR_CUDA;
    if (e == cudaSuccess) {
        ctx->graph_capturing = true;
        st = issue_fdpf(ctx, opts, vm_dev, va_dev, engine, ctx->gstream);
        ctx->graph_capturing = false;
        e = cudaStreamEndCapture(ctx->gstream, &graph);
    }
    if (e == cudaSuccess && st == PF_OK) e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || st != PF_OK) {  // no graphs for this context: run directly
        cudaGetLastError();
        ctx->gexec = nullptr;
        ctx->graphs_off = true;
        return issue_fdpf(ctx, opts, vm_dev, va_dev, engine, s);
    }
    ctx->gkey = key;
    e = cudaGraphLaunch(ctx->gexec, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
    for (int q = 0; q < PF_K_COUNT; q++) ctx->kstat[q].launches += ctx->glaunches[q];
    return PF_OK;
}

pf_status run_once(pf_ctx *ctx, const pf_run_opts *opts, double *vm_dev, double *va_dev,
                   pf_case_result *res_host, void *stream) {
    if (!ctx || !opts || !vm_dev || !va_dev || !res_host) return fail(ctx, PF_ERR_ARG, "null pointer");
    if (!ctx->analyzed) return fail(ctx, PF_ERR_STATE, "pf_analyze first");
    if (opts->method != PF_FDPF && opts->method != PF_NR)
        return fail(ctx, PF_ERR_ARG, "method %d not available", opts->method);
    if (opts->precision != PF_FP64 && opts->precision != PF_FP32)
        return fail(ctx, PF_ERR_ARG, "bad precision");
    if (!(opts->tol > 0) || opts->max_iter < 1) return fail(ctx, PF_ERR_ARG, "bad tol/max_iter");
    if (opts->precision == PF_FP32 && (opts->ir_max < 0 || opts->ir_max > 100 || !(opts->ir_tol >= 0)))
        return fail(ctx, PF_ERR_ARG, "bad refinement options");
    TRY(ensure_cases(ctx));
    cudaStream_t s = (cudaStream_t)stream;
    const int prec = opts->precision;
    if (opts->method == PF_NR) {
        TRY(assemble_ybus(ctx, s));
        TRY(ensure_nr_storage(ctx, prec));
        NrLaunch L = nr_launch(ctx, prec);
        L.o = *opts;
        L.vm = vm_dev;
        L.va = va_dev;
        L.epoch0 = nr_epochs(ctx, unsigned(opts->max_iter) + 2u, s);
        cudaError_t e = counted(ctx, PF_K_RUN, 1, s, [&] { return launch_nr(L, s); });
        if (e != cudaSuccess) return cuda_fail(ctx, e, "nr launch");
        ctx->ws.jfactored[prec] = true;
        e = cudaMemcpyAsync(res_host, ctx->ws.res, sizeof(pf_case_result) * ctx->dc.ncase,
                            cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "nr run");
        for (int c = 0; c < ctx->dc.ncase; c++)
            if (res_host[c].status != PF_OK)
                return fail(ctx, pf_status(res_host[c].status), "case %d: status %d after %d iterations",
                            c, res_host[c].status, res_host[c].iters);
        return PF_OK;
    }
    Workspace &w = ctx->ws;
    const int nmax = std::max(ctx->dm[0].n, ctx->dm[1].n);
    // the lane engine has no Newton-Raphson fallback: runs that ask for it use the others
    const bool lanes_ok = opts->method == PF_FDPF && !opts->fallback && lane_width(nmax, prec, ctx->smem_optin) > 0;
    const int want = opts->engine != PF_ENGINE_AUTO ? opts->engine : ctx->tune.engine;
    const bool use_cluster = want == PF_ENGINE_CLUSTER && cluster_applies(ctx, opts);
    const int engine = use_cluster ? PF_ENGINE_CLUSTER
                                   : (want == PF_ENGINE_LANES && lanes_ok ? PF_ENGINE_LANES : PF_ENGINE_BLOCK);
    if (engine == PF_ENGINE_LANES) {
        TRY(assemble_ybus(ctx, s));
        TRY(factor_both(ctx, prec, s, false));
        const void *F0 = prec == PF_FP64 ? (const void *)w.F64[0] : (const void *)w.F32[0];
        const void *F1 = prec == PF_FP64 ? (const void *)w.F64[1] : (const void *)w.F32[1];
        TRY(ensure_lanes(ctx, prec));
        LaneRun r;
        r.dn = ctx->dn;
        r.dc = ctx->dc;
        r.m0 = ctx->dm[0];
        r.m1 = ctx->dm[1];
        r.L = ctx->ws.lanes;
        r.F0 = F0;
        r.F1 = F1;
        r.fs0 = w.fstatus[0][prec];
        r.fs1 = w.fstatus[1][prec];
        r.A0 = w.A[0];
        r.A1 = w.A[1];
        r.o = *opts;
        r.prec = prec;
        r.vm = vm_dev;
        r.va = va_dev;
        r.res = w.res;
        r.smem_optin = ctx->smem_optin;
        cudaError_t e = counted(ctx, PF_K_RUN, 1, s, [&] { return lane_run(r, s); });
        if (e != cudaSuccess) return cuda_fail(ctx, e, "lane engine");
        e = cudaMemcpyAsync(res_host, w.res, sizeof(pf_case_result) * ctx->dc.ncase,
                            cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "lane engine");
        for (int c = 0; c < ctx->dc.ncase; c++)
            if (res_host[c].status != PF_OK)
                return fail(ctx, pf_status(res_host[c].status), "case %d: status %d after %d iterations",
                            c, res_host[c].status, res_host[c].iters);
        return PF_OK;
    }
    // block and cluster engines: the device work of the run (the admittance
    // matrix first), enqueued directly or from a CUDA graph of it
    TRY(run_device_work(ctx, opts, vm_dev, va_dev, engine, s));
    cudaError_t e = cudaMemcpyAsync(res_host, w.res, sizeof(pf_case_result) * ctx->dc.ncase,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fdpf run");
    for (int c = 0; c < ctx->dc.ncase; c++)
        if (res_host[c].status != PF_OK)
            return fail(ctx, pf_status(res_host[c].status), "case %d: status %d after %d iterations (%s)",
                        c, res_host[c].status, res_host[c].iters, res_host[c].method == PF_NR ? "NR" : "FDPF");
    return PF_OK;
}

}  // namespace

extern "C" {

pf_status pf_adjoint(pf_ctx *ctx, int32_t precision, const double *vm_dev, const double *va_dev,
                     const double *gva_dev, const double *gvm_dev, double *dJdP_dev,
                     double *dJdQ_dev, pf_case_result *res_host, void *stream) {
    if (!ctx || !vm_dev || !va_dev || !gva_dev || !gvm_dev || !dJdP_dev || !dJdQ_dev || !res_host ||
        (precision != PF_FP64 && precision != PF_FP32))
        return fail(ctx, PF_ERR_ARG, "bad argument");
    if (!ctx->analyzed) return fail(ctx, PF_ERR_STATE, "pf_analyze first");
    TRY(ensure_cases(ctx));
    cudaStream_t s = (cudaStream_t)stream;
    TRY(assemble_ybus(ctx, s));
    TRY(ensure_nr_storage(ctx, precision));
    NrLaunch L = nr_launch(ctx, precision);
    L.o.tol = 1e-8;
    L.o.ir_max = 20;
    L.o.ir_tol = 1e-14;
    L.o.ir_abs = 1e-300;
    L.vm = const_cast<double *>(vm_dev);
    L.va = const_cast<double *>(va_dev);
    L.gva = gva_dev;
    L.gvm = gvm_dev;
    L.dJdP = dJdP_dev;
    L.dJdQ = dJdQ_dev;
    L.adjoint = true;
    L.factor_now = ctx->ws.jfactored[precision] ? 0 : 1;
    L.epoch0 = nr_epochs(ctx, 2u, s);
    cudaError_t e = counted(ctx, PF_K_RUN, 1, s, [&] { return launch_nr(L, s); });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint launch");
    ctx->ws.jfactored[precision] = true;
    e = cudaMemcpyAsync(res_host, ctx->ws.res, sizeof(pf_case_result) * ctx->dc.ncase,
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint");
    for (int c = 0; c < ctx->dc.ncase; c++)
        if (res_host[c].status != PF_OK)
            return fail(ctx, pf_status(res_host[c].status), "adjoint case %d: status %d", c,
                        res_host[c].status);
    return PF_OK;
}

pf_status pf_objective(pf_ctx *ctx, const double *vm_dev, const double *va_dev, double *J_dev,
                       double *gva_dev, double *gvm_dev, void *stream) {
    if (!ctx || !vm_dev || !va_dev || !J_dev || !gva_dev || !gvm_dev)
        return fail(ctx, PF_ERR_ARG, "null pointer");
    if (!ctx->analyzed) return fail(ctx, PF_ERR_STATE, "pf_analyze first");
    TRY(ensure_cases(ctx));
    cudaStream_t s = (cudaStream_t)stream;
    TRY(assemble_ybus(ctx, s));
    cudaError_t e = counted(ctx, PF_K_MISMATCH, 1, s, [&] {
        return launch_objective(ctx->dn, ctx->dc, vm_dev, va_dev, ctx->ws.ef, J_dev, gva_dev, gvm_dev, s);
    });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "objective launch");
    return PF_OK;
}

pf_status pf_set_graphs(pf_ctx *ctx, int32_t on) {
    if (!ctx) return PF_ERR_ARG;
    drop_graph(ctx);
    ctx->graphs_off = !on;
    return PF_OK;
}

pf_status pf_set_profiling(pf_ctx *ctx, int32_t on) {
    if (!ctx) return PF_ERR_ARG;
    ctx->profiling = on != 0;
    return PF_OK;
}

pf_status pf_get_profile(pf_ctx *ctx, int32_t kind, int64_t *launches, double *total_ms,
                         int32_t reset) {
    if (!ctx || kind < 0 || kind >= PF_K_COUNT) return PF_ERR_ARG;
    KernelStat &k = ctx->kstat[kind];
    drain_events(ctx, k);
    if (launches) *launches = k.launches;
    if (total_ms) *total_ms = k.ms;
    if (reset) {
        k.launches = 0;
        k.ms = 0.0;
    }
    return PF_OK;
}

const char *pf_last_error(const pf_ctx *ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

pf_status pf_get_ybus(pf_ctx *ctx, int32_t *rowptr, int32_t *col, double *G, double *B) {
    if (!ctx) return PF_ERR_ARG;
    if (rowptr) std::copy(ctx->rowptr.begin(), ctx->rowptr.end(), rowptr);
    if (col) std::copy(ctx->col.begin(), ctx->col.end(), col);
    if (G || B) {
        TRY(ensure_device(ctx));
        TRY(assemble_ybus(ctx, 0));
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess && G)
            e = cudaMemcpy(G, ctx->dn.G, sizeof(double) * ctx->dn.nnz, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && B)
            e = cudaMemcpy(B, ctx->dn.B, sizeof(double) * ctx->dn.nnz, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "get_ybus");
    }
    return PF_OK;
}

pf_status pf_branch_flows(pf_ctx *ctx, const double *vm_dev, const double *va_dev, int32_t ncase,
                          double *flows_dev, double *loss_dev, void *stream) {
    if (!ctx || !vm_dev || !va_dev || !flows_dev || !loss_dev) return fail(ctx, PF_ERR_ARG, "null pointer");
    TRY(ensure_cases(ctx));
    if (ncase < 1 || ncase > ctx->dc.ncase) return fail(ctx, PF_ERR_ARG, "ncase out of range");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = counted(ctx, PF_K_MISMATCH, 2, s, [&] {
        return launch_branch_flows(ctx->dn, ctx->dc, vm_dev, va_dev, ncase, flows_dev, loss_dev, s);
    });
    if (e != cudaSuccess) return cuda_fail(ctx, e, "branch flows launch");
    return PF_OK;
}

pf_status pf_get_tuning(const pf_ctx *ctx, pf_tuning *out) {
    if (!ctx || !out) return PF_ERR_ARG;
    *out = ctx->tune;
    return PF_OK;
}

pf_status pf_set_tuning(pf_ctx *ctx, const pf_tuning *t) {
    if (!ctx || !t) return fail(ctx, PF_ERR_ARG, "null pointer");
    const bool cl_engine = t->engine == PF_ENGINE_CLUSTER;
    if (t->engine < 0 || t->engine > PF_ENGINE_CLUSTER || t->factor < 0 || t->factor > 2 || t->tail < 0 ||
        t->tail > 3 || t->outage < 0 || t->outage > 2 ||
        (!cl_engine && t->cluster != 0 && t->cluster != 1 && t->cluster != 8 && t->cluster != 16) ||
        (cl_engine && (t->cluster < 0 || t->cluster > kClGroupMax)) ||
        (t->threads != 0 && t->threads != 128 && t->threads != 256 && t->threads != 512))
        return fail(ctx, PF_ERR_ARG, "tuning field out of range");
    ctx->tune = *t;
    ctx->tune.ms = t->ms;
    if (cl_engine && ctx->analyzed) TRY(set_cluster_group(ctx, t->cluster > 0 ? t->cluster : kClGroupDefault));
    return PF_OK;
}

pf_status pf_autotune(pf_ctx *ctx, const pf_run_opts *opts, double *vm_dev, double *va_dev,
                      int32_t reps, pf_tuning *out, void *stream) {
    if (!ctx || !opts || !vm_dev || !va_dev || !out) return fail(ctx, PF_ERR_ARG, "null pointer");
    if (reps < 1 || reps > 1000) return fail(ctx, PF_ERR_ARG, "reps out of range");
    if (!ctx->analyzed) return fail(ctx, PF_ERR_STATE, "pf_analyze first");
    TRY(ensure_cases(ctx));
    TRY(ensure_device(ctx));
    cudaStream_t s = (cudaStream_t)stream;
    pf_run_opts o = *opts;
    o.engine = PF_ENGINE_AUTO;
    const int ncase = ctx->dc.ncase;
    const int prec = o.precision;
    // candidate mappings
    std::vector<pf_tuning> cand;
    std::vector<int> engines{PF_ENGINE_BLOCK};
    const int nmax = std::max(ctx->dm[0].n, ctx->dm[1].n);
    if (o.method == PF_FDPF && ncase >= 32 && lane_width(nmax, prec, ctx->smem_optin) > 0)
        engines.push_back(PF_ENGINE_LANES);
    if (cluster_applies(ctx, &o)) engines.push_back(PF_ENGINE_CLUSTER);
    std::vector<int> clusters{0};
    if (o.method == PF_FDPF) {
        const int cmax = fdpf_cluster_size(ncase, ctx->num_sms, prec, ctx->smem_optin, nmax);
        clusters.clear();
        for (int c : {1, 8, 16})
            if (c <= cmax) clusters.push_back(c);
    }
    std::vector<int> factors{2};
    if (std::max(ctx->hm[0].max_col, ctx->hm[1].max_col) <= kDepMaxCol) factors.push_back(1);
    std::vector<int> tails{2};
    if (o.method == PF_FDPF && (ctx->dm[0].npf2 > 0 || ctx->dm[1].npf2 > 0)) tails.push_back(1);
    if (o.method == PF_FDPF && (ctx->dm[0].npf3 > 0 || ctx->dm[1].npf3 > 0)) tails.push_back(3);
    std::vector<int> outages{1};
    if (o.method == PF_FDPF && ctx->dc.ninst > 1) outages.push_back(2);
    // the lane engine has no cluster, tail or outage choice; the cluster
    // engine no cluster size (its own) and no outage form (one base case)
    // block sizes matter only for one block per case of a batch
    // the cluster engine's field `cluster` is its subtree levels per step
    for (int e : engines)
        for (int c : (e == PF_ENGINE_CLUSTER ? std::vector<int>{1, 2, 3, 4}
                                             : (e != PF_ENGINE_BLOCK ? std::vector<int>{0} : clusters)))
            for (int f : factors)
                for (int t : (e == PF_ENGINE_LANES ? std::vector<int>{0} : tails))
                    for (int u : (e != PF_ENGINE_BLOCK ? std::vector<int>{1} : outages))
                        for (int th : (e == PF_ENGINE_BLOCK && c == 1 && ncase > 1 ? std::vector<int>{512, 256, 128}
                                                                                    : std::vector<int>{0})) {
                            // tail form 3 serves runs whose solves all use instance 0, on the block engine
                            if (t == 3 && (e != PF_ENGINE_BLOCK || (ctx->dc.ninst > 1 && u != 2))) continue;
                            cand.push_back(pf_tuning{e, c, f, t, u, th, 0.0});
                        }
    std::vector<pf_case_result> res(static_cast<size_t>(ncase));
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return fail(ctx, PF_ERR_CUDA, "event creation");
    }
    const pf_tuning saved = ctx->tune;
    const bool graphs_saved = ctx->graphs_off;
    ctx->graphs_off = true;  // every candidate timed on direct launches
    pf_tuning best{0, 0, 0, 0, 0, 0, -1.0};
    pf_status last = PF_OK;
    for (const pf_tuning &t : cand) {
        ctx->tune = t;
        if (t.engine == PF_ENGINE_CLUSTER) TRY(set_cluster_group(ctx, t.cluster > 0 ? t.cluster : kClGroupDefault));
        pf_status st = pf_run_to_tol(ctx, &o, vm_dev, va_dev, res.data(), stream);  // untimed
        if (st != PF_OK) {
            last = st;
            continue;
        }
        cudaEventRecord(a, s);
        for (int r = 0; r < reps && st == PF_OK; r++) st = pf_run_to_tol(ctx, &o, vm_dev, va_dev, res.data(), stream);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (st != PF_OK) {
            last = st;
            continue;
        }
        const double per = double(ms) / reps;
        if (best.ms < 0 || per < best.ms) {
            best = t;
            best.ms = per;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->graphs_off = graphs_saved;
    if (best.ms < 0) {
        ctx->tune = saved;
        return fail(ctx, last == PF_OK ? PF_ERR_NOT_CONVERGED : last, "no mapping converged");
    }
    ctx->tune = best;
    if (best.engine == PF_ENGINE_CLUSTER)
        TRY(set_cluster_group(ctx, best.cluster > 0 ? best.cluster : kClGroupDefault));
    *out = best;
    return PF_OK;
}

}  // extern "C"

struct pf_pack {
    std::vector<pf_ctx *> grids;
    std::vector<int> order;       // grids by decreasing size
    std::vector<int64_t> offset;  // first bus of each grid in the concatenated state
    std::vector<int2> items;      // factor work items (job = 2 grid + matrix, column)
    int2 *items_dev = nullptr;
    gbpf::FactorJob *jobs_dev = nullptr;
    unsigned *fsync = nullptr;
    void *args = nullptr;
    int *order_dev = nullptr;
    unsigned *counter = nullptr;
    pf_case_result *res = nullptr;
    int device = 0, num_sms = 0;
    size_t smem_optin = 0;
    std::string err;
};

namespace {
pf_status pack_fail(pf_pack *pk, pf_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (pk) pk->err = buf;
    return st;
}
}  // namespace

extern "C" {

pf_status pf_pack_create(pf_ctx *const *grids, int32_t ngrid, pf_pack **out) {
    if (!out) return PF_ERR_ARG;
    *out = nullptr;
    if (!grids || ngrid < 1) return PF_ERR_ARG;
    auto *pk = new (std::nothrow) pf_pack();
    if (!pk) return PF_ERR_OOM;
    std::vector<pf_ctx *> seen;
    int64_t off = 0;
    for (int g = 0; g < ngrid; g++) {
        pf_ctx *c = grids[g];
        if (!c || std::find(seen.begin(), seen.end(), c) != seen.end()) {
            delete pk;
            return PF_ERR_ARG;
        }
        if (!c->analyzed) {
            delete pk;
            return PF_ERR_STATE;
        }
        if (c->hm[0].max_col > gbpf::kDepMaxCol || c->hm[1].max_col > gbpf::kDepMaxCol) {
            delete pk;  // a column longer than the packed factor takes
            return PF_ERR_ARG;
        }
        seen.push_back(c);
        pk->grids.push_back(c);
        pk->offset.push_back(off);
        off += c->nbus;
    }
    pk->order.resize(size_t(ngrid));
    for (int g = 0; g < ngrid; g++) pk->order[g] = g;
    std::stable_sort(pk->order.begin(), pk->order.end(), [&](int a, int b) {
        return pk->grids[a]->nbus > pk->grids[b]->nbus;
    });
    // factor work items: levels ascending across all matrices, so every
    // column follows the columns it depends on
    int maxlev = 0;
    for (pf_ctx *c : pk->grids)
        for (int w = 0; w < 2; w++) maxlev = std::max(maxlev, c->hm[w].nlev);
    for (int l = 0; l < maxlev; l++)
        for (int g = 0; g < ngrid; g++)
            for (int w = 0; w < 2; w++) {
                const gbpf::HostMat &H = pk->grids[g]->hm[w];
                if (l >= H.nlev) continue;
                for (int c = H.lvl_ptr[l]; c < H.lvl_ptr[l + 1]; c++) pk->items.push_back(int2{2 * g + w, c});
            }
    *out = pk;
    return PF_OK;
}

pf_status pf_pack_run(pf_pack *pk, const pf_run_opts *opts, double *vm_dev, double *va_dev,
                      pf_case_result *res_host, void *stream) {
    if (!pk || !opts || !vm_dev || !va_dev || !res_host) return pack_fail(pk, PF_ERR_ARG, "null pointer");
    if (opts->method != PF_FDPF) return pack_fail(pk, PF_ERR_ARG, "packs run the fast decoupled method");
    if (opts->precision != PF_FP64 && opts->precision != PF_FP32)
        return pack_fail(pk, PF_ERR_ARG, "bad precision");
    if (!(opts->tol > 0) || opts->max_iter < 1) return pack_fail(pk, PF_ERR_ARG, "bad tol/max_iter");
    if (opts->precision == PF_FP32 && (opts->ir_max < 0 || opts->ir_max > 100 || !(opts->ir_tol >= 0)))
        return pack_fail(pk, PF_ERR_ARG, "bad refinement options");
    const int ngrid = int(pk->grids.size());
    const int prec = opts->precision;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<PackGrid> pg(static_cast<size_t>(ngrid));
    std::vector<FactorJob> jobs(static_cast<size_t>(2 * ngrid));
    for (int g = 0; g < ngrid; g++) {
        pf_ctx *ctx = pk->grids[g];
        pf_status st = ensure_cases(ctx);
        if (st == PF_OK && ctx->dc.ncase != 1) st = fail(ctx, PF_ERR_STATE, "a packed grid has one case");
        if (st == PF_OK) st = assemble_ybus(ctx, s);
        if (st == PF_OK) st = assemble_matrix(ctx, PF_MAT_BP, prec, s);
        if (st == PF_OK) st = assemble_matrix(ctx, PF_MAT_BPP, prec, s);
        if (st == PF_OK) st = factor_job(ctx, PF_MAT_BP, prec, jobs[2 * g], s);
        if (st == PF_OK) st = factor_job(ctx, PF_MAT_BPP, prec, jobs[2 * g + 1], s);
        if (st != PF_OK) return pack_fail(pk, st, "grid %d: %s", g, ctx->err.c_str());
        Workspace &w = ctx->ws;
        PackGrid &p = pg[g];
        p.dn = ctx->dn;
        p.dc = ctx->dc;
        p.m[0] = ctx->dm[0];
        p.m[1] = ctx->dm[1];
        p.F0 = prec == PF_FP64 ? (const void *)w.F64[0] : (const void *)w.F32[0];
        p.F1 = prec == PF_FP64 ? (const void *)w.F64[1] : (const void *)w.F32[1];
        p.TV0 = ctx->tune.tail != 2 ? w.TV[0][prec] : nullptr;
        p.TV1 = ctx->tune.tail != 2 ? w.TV[1][prec] : nullptr;
        p.A0 = w.A[0];
        p.A1 = w.A[1];
        p.fs0 = w.fstatus[0][prec];
        p.fs1 = w.fstatus[1][prec];
        p.vm = vm_dev + pk->offset[g];
        p.va = va_dev + pk->offset[g];
        p.ef = w.ef;
        p.iv = w.iv;
        p.xg = w.vec;
        p.bmax = w.bmax;
        p.res = nullptr;  // set below
        if (g == 0) {
            pk->device = ctx->device;
            pk->num_sms = ctx->num_sms;
            pk->smem_optin = ctx->smem_optin;
        } else if (ctx->device != pk->device) {
            return pack_fail(pk, PF_ERR_ARG, "grid %d is on another device", g);
        }
    }
    cudaError_t e = cudaSuccess;
    if (!pk->args) {
        e = cudaMalloc(reinterpret_cast<void **>(&pk->jobs_dev), sizeof(FactorJob) * size_t(2 * ngrid));
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&pk->fsync), 2 * sizeof(unsigned));
        if (e == cudaSuccess)
            e = cudaMalloc(reinterpret_cast<void **>(&pk->items_dev), sizeof(int2) * std::max<size_t>(1, pk->items.size()));
        if (e == cudaSuccess)
            e = cudaMemcpy(pk->items_dev, pk->items.data(), sizeof(int2) * pk->items.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&pk->args, run_args_bytes() * size_t(ngrid));
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&pk->order_dev), sizeof(int) * size_t(ngrid));
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&pk->counter), sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&pk->res), sizeof(pf_case_result) * size_t(ngrid));
        if (e != cudaSuccess)
            return pack_fail(pk, e == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA, "pack scratch: %s",
                             cudaGetErrorString(e));
    }
    for (int g = 0; g < ngrid; g++) pg[g].res = pk->res + g;
    // every grid's B' and B'' in one factor launch
    e = cudaMemcpyAsync(pk->jobs_dev, jobs.data(), sizeof(FactorJob) * jobs.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // jobs is released on return
    if (e == cudaSuccess)
        e = launch_factor_jobs(pk->jobs_dev, 2 * ngrid, pk->items_dev, unsigned(pk->items.size()), pk->fsync,
                               prec, pk->num_sms, s);
    if (e != cudaSuccess)
        return pack_fail(pk, e == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA, "pack factor: %s",
                         cudaGetErrorString(e));
    for (pf_ctx *ctx : pk->grids)
        for (int w = 0; w < 2; w++) ctx->ws.factored[w][prec] = true;
    e = launch_pack(pg.data(), ngrid, prec, *opts, pk->order.data(), pk->args, pk->order_dev, pk->counter,
                    pk->smem_optin, pk->num_sms, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res_host, pk->res, sizeof(pf_case_result) * size_t(ngrid), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return pack_fail(pk, e == cudaErrorMemoryAllocation ? PF_ERR_OOM : PF_ERR_CUDA, "pack run: %s",
                         cudaGetErrorString(e));
    for (int g = 0; g < ngrid; g++)
        if (res_host[g].status != PF_OK)
            return pack_fail(pk, pf_status(res_host[g].status), "grid %d: status %d after %d iterations", g,
                             res_host[g].status, res_host[g].iters);
    return PF_OK;
}

const char *pf_pack_last_error(const pf_pack *pk) { return pk ? pk->err.c_str() : "null pack"; }

void pf_pack_destroy(pf_pack *pk) {
    if (!pk) return;
    cudaFree(pk->args);
    cudaFree(pk->jobs_dev);
    cudaFree(pk->items_dev);
    cudaFree(pk->fsync);
    cudaFree(pk->order_dev);
    cudaFree(pk->counter);
    cudaFree(pk->res);
    delete pk;
}

void pf_destroy(pf_ctx *ctx) {
    if (!ctx) return;
    drop_graph(ctx);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    if (ctx->ws.side) {
        cudaStreamSynchronize(ctx->ws.side);
        cudaStreamDestroy(ctx->ws.side);
        cudaEventDestroy(ctx->ws.fork);
        cudaEventDestroy(ctx->ws.join);
    }
    for (auto &k : ctx->kstat) {
        for (auto &pr : k.pending) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        k.pending.clear();
    }
    for (void *p : ctx->allocations) cudaFree(p);
    ctx->allocations.clear();
    delete ctx;
}

// Test hook (host only, no GPU needed): the tail-factor tables of matrix
// `which` (0 = B', 1 = B'') as built by pf_analyze.  sizes[8] receives {n,
// t0, ntl, ng, ne, kmax, tmax, number of tail terms}; tlev (4 ints per
// entry, 2 ntl entries) and tinfo (4 ints per target, ng targets) are copied
// when cap_lev >= 2 ntl and cap_tgt >= ng.  Returns 0, or -1 for a bad
// argument or a matrix that has not been analysed.
int gbpf_debug_tail_tables(const pf_ctx *ctx, int which, int *sizes, int *tlev, int cap_lev,
                           int *tinfo, int cap_tgt) {
    if (!ctx || !sizes || which < 0 || which > 1) return -1;
    const gbpf::HostMat &H = ctx->hm[which];
    if (H.lvl_ptr.empty()) return -1;
    const int ntail = H.tptr.empty() ? 0 : H.tptr.back();
    const int v[8] = {H.n, H.t0, H.ntl, H.ft_ng, H.ft_ne, H.ft_kmax, H.ft_tmax, ntail};
    for (int i = 0; i < 8; i++) sizes[i] = v[i];
    if (tlev && cap_lev >= 2 * H.ntl)
        for (int i = 0; i < 2 * H.ntl; i++) {
            const int4 e = H.tlev[size_t(i)];
            tlev[4 * i] = e.x, tlev[4 * i + 1] = e.y, tlev[4 * i + 2] = e.z, tlev[4 * i + 3] = e.w;
        }
    if (tinfo && cap_tgt >= H.ft_ng)
        for (int i = 0; i < H.ft_ng; i++) {
            const int4 e = H.tinfo[size_t(i)];
            tinfo[4 * i] = e.x, tinfo[4 * i + 1] = e.y, tinfo[4 * i + 2] = e.z, tinfo[4 * i + 3] = e.w;
        }
    return 0;
}

// Test hook (host only, no GPU needed): the scatter-tail schedules of matrix
// `which` as built by pf_analyze.  sizes[6] receives {t0, ntl, len(SKf),
// len(SIf), len(SKb), len(SIb)}; the four arrays are copied when cap (ints
// per array) covers them.  Returns 0, or -1 for a bad argument or a matrix
// that has not been analysed.
int gbpf_debug_scatter_schedules(const pf_ctx *ctx, int which, int *sizes, int *SKf, int *SIf,
                                 int *SKb, int *SIb, int cap) {
    if (!ctx || !sizes || which < 0 || which > 1) return -1;
    const gbpf::HostMat &H = ctx->hm[which];
    if (H.lvl_ptr.empty()) return -1;
    const int v[6] = {H.t0, H.ntl, int(H.SKf.size()), int(H.SIf.size()), int(H.SKb.size()),
                      int(H.SIb.size())};
    for (int i = 0; i < 6; i++) sizes[i] = v[i];
    const std::vector<int> *src[4] = {&H.SKf, &H.SIf, &H.SKb, &H.SIb};
    int *dst[4] = {SKf, SIf, SKb, SIb};
    for (int a = 0; a < 4; a++)
        if (dst[a] && cap >= int(src[a]->size())) std::copy(src[a]->begin(), src[a]->end(), dst[a]);
    return 0;
}

// Test hook (host only, no GPU needed): a piece list of matrix `which`
// (list 0 = forward sweep, 1 = backward sweep, 2 / 3 = the same with a
// scatter tail) as 8 ints per piece {r0, r1, e0, e1, mode, run_end, l0, l1};
// *count receives the number of pieces, copied when cap >= 8 * count.
// Returns 0, or -1 for a bad argument or a matrix that has not been analysed.
int gbpf_debug_pieces(const pf_ctx *ctx, int which, int list, int *count, int *out, int cap) {
    if (!ctx || !count || which < 0 || which > 1 || list < 0 || list > 3) return -1;
    const gbpf::HostMat &H = ctx->hm[which];
    if (H.lvl_ptr.empty()) return -1;
    const std::vector<gbpf::Piece> *L[4] = {&H.pf, &H.pb, &H.pf2, &H.pb2};
    const std::vector<gbpf::Piece> &P = *L[list];
    *count = int(P.size());
    if (out && cap >= 8 * int(P.size()))
        for (size_t i = 0; i < P.size(); i++) {
            const gbpf::Piece &q = P[i];
            const int v[8] = {q.r0, q.r1, q.e0, q.e1, q.mode, q.run_end, q.l0, q.l1};
            std::copy(v, v + 8, out + 8 * i);
        }
    return 0;
}

// Test hook (host only, no GPU needed): the level-order CSC pattern of L and
// the gather lists of the dependency-driven factor of matrix `which`.
// sizes[3] receives {n, nnz (strict lower), number of gather terms}; Cp (n + 1),
// Cr (nnz), gp (n + nnz + 1) and gl (4 ints per term) are copied when cap (ints
// per array) covers them.  Returns 0, or -1 for a bad argument or a matrix
// that has not been analysed.
// Test hook (host only, no GPU needed): the admittance assembly's per-entry
// tables and the mismatch's thread orders.  sizes[3] receives {nbus, nnz,
// off-diagonal entries, branch references}; when cap (ints per array)
// covers them, rowptr (nbus + 1), col (nnz), yoff (4 per off-diagonal
// entry), yoff_br, mis_ord and mis_ord_cl (nbus each) are copied.  Returns
// 0, or -1 for a bad argument.
int gbpf_debug_net_tables(const pf_ctx *ctx, long long *sizes, int *rowptr, int *col, int *yoff, int *yoff_br,
                          int *mis_ord, int *mis_ord_cl, long long cap) {
    if (!ctx || !sizes) return -1;
    sizes[0] = ctx->nbus;
    sizes[1] = (long long)ctx->col.size();
    sizes[2] = (long long)ctx->yoff.size();
    sizes[3] = (long long)ctx->yoff_br.size();
    if (rowptr && cap > ctx->nbus) std::copy(ctx->rowptr.begin(), ctx->rowptr.end(), rowptr);
    if (col && cap >= sizes[1]) std::copy(ctx->col.begin(), ctx->col.end(), col);
    if (yoff && cap >= 4 * sizes[2])
        for (size_t k = 0; k < ctx->yoff.size(); k++) {
            yoff[4 * k] = ctx->yoff[k].x;
            yoff[4 * k + 1] = ctx->yoff[k].y;
            yoff[4 * k + 2] = ctx->yoff[k].z;
            yoff[4 * k + 3] = ctx->yoff[k].w;
        }
    if (yoff_br && cap >= sizes[3]) std::copy(ctx->yoff_br.begin(), ctx->yoff_br.end(), yoff_br);
    if (mis_ord && cap >= ctx->nbus) std::copy(ctx->mis_ord.begin(), ctx->mis_ord.end(), mis_ord);
    if (mis_ord_cl && cap >= ctx->nbus) std::copy(ctx->mis_ord_cl.begin(), ctx->mis_ord_cl.end(), mis_ord_cl);
    return 0;
}

int gbpf_debug_gather(const pf_ctx *ctx, int which, long long *sizes, int *Cp, int *Cr, int *gp,
                      int *gl, long long cap) {
    if (!ctx || !sizes || which < 0 || which > 1) return -1;
    const gbpf::HostMat &H = ctx->hm[which];
    if (H.lvl_ptr.empty() || H.Cp.empty()) return -1;
    const long long nnz = H.Cp.back();
    const long long nterm = H.gp.empty() ? 0 : H.gp.back();
    sizes[0] = H.n;
    sizes[1] = nnz;
    sizes[2] = nterm;
    if (Cp && cap >= (long long)H.Cp.size()) std::copy(H.Cp.begin(), H.Cp.end(), Cp);
    if (Cr && cap >= nnz) std::copy(H.Cr.begin(), H.Cr.begin() + nnz, Cr);
    if (gp && cap >= (long long)H.gp.size()) std::copy(H.gp.begin(), H.gp.end(), gp);
    if (gl && cap >= 4 * nterm)
        for (long long q = 0; q < nterm; q++) {
            const int4 e = H.gl[size_t(q)];
            gl[4 * q] = e.x, gl[4 * q + 1] = e.y, gl[4 * q + 2] = e.z, gl[4 * q + 3] = e.w;
        }
    return 0;
}

// Test hook (host only, no GPU needed): the cluster engine's program of
// matrix `which`.  sizes[12] receives {C, nt, steps (all CTAs), nx, tasks,
// entries, values, dynamic shared memory of a CTA, offDi, offLc, offLr, ok};
// the arrays are copied when cap (ints per array) covers them: tasks, steps
// and vsrc (4 ints each), tptr, eptr, vptr, sptr (C + 1), refs, rhsref and
// xref (nbus), tnode (nt: the level-order rows of the top set).  Returns 0, or -1 for a bad argument
// or a context that has not been analysed.
int gbpf_debug_cluster(const pf_ctx *ctx, int which, long long *sizes, int *tasks, int *tptr,
                       int *steps, int *refs, int *eptr, int *vsrc, int *vptr, int *sptr, int *rhsref,
                       int *xref, int *tnode, long long cap) {
    if (!ctx || !sizes || which < 0 || which > 1 || !ctx->analyzed) return -1;
    const gbpf::HostCl &P = ctx->hcl[which];
    const gbpf::HostMat &H = ctx->hm[which];
    const long long v[12] = {gbpf::kClCtas, P.nt, (long long)P.steps.size(), P.nx, (long long)P.tasks.size(),
                             (long long)P.refs.size(), (long long)P.vsrc.size(), (long long)ctx->cl_smem,
                             H.offDi, H.offLc, H.offLr, P.ok};
    for (int i = 0; i < 12; i++) sizes[i] = v[i];
    auto put4 = [&](const std::vector<int4> &a, int *dst) {
        if (dst && cap >= 4 * (long long)a.size())
            for (size_t i = 0; i < a.size(); i++) {
                dst[4 * i] = a[i].x, dst[4 * i + 1] = a[i].y, dst[4 * i + 2] = a[i].z, dst[4 * i + 3] = a[i].w;
            }
    };
    auto put = [&](const std::vector<int> &a, int *dst) {
        if (dst && cap >= (long long)a.size()) std::copy(a.begin(), a.end(), dst);
    };
    put4(P.tasks, tasks);
    put(P.tptr, tptr);
    put4(P.steps, steps);
    put(P.refs, refs);
    put(P.eptr, eptr);
    put4(P.vsrc, vsrc);
    put(P.vptr, vptr);
    put(P.sptr, sptr);
    put(P.rhsref, rhsref);
    put(P.xref, xref);
    put(P.tnode, tnode);
    return 0;
}

// Test hook (host only, no GPU needed): the grouped subtree steps' value
// programs of matrix `which` in the cluster engine.  sizes[6] receives
// {group, inverse columns, inverse entries, combined entries, updates,
// terms}; gw_col and gw_upd (4 ints each), gm_ptr (combined entries + 1),
// gm_term (2 ints each) and gv_info (4 ints per value) are copied when cap
// (ints per array) covers them.  Returns 0, or -1 for a bad argument or a
// context that has not been analysed.
int gbpf_debug_cluster_groups(const pf_ctx *ctx, int which, int *sizes, int *gw_col, int *gw_upd, int *gm_ptr,
                              int *gm_term, int *gv_info, long long cap) {
    if (!ctx || !sizes || which < 0 || which > 1 || !ctx->analyzed) return -1;
    const gbpf::HostCl &P = ctx->hcl[which];
    sizes[0] = P.group;
    sizes[1] = P.n_gwcol;
    sizes[2] = P.n_gw;
    sizes[3] = P.n_gm;
    sizes[4] = P.n_gwcol > 0 ? int(P.gw_upd.size()) : 0;
    sizes[5] = P.n_gm > 0 ? P.gm_ptr.back() : 0;
    auto put4 = [&](const std::vector<int4> &a, size_t count, int *dst) {
        if (dst && cap >= 4 * (long long)count)
            for (size_t i = 0; i < count; i++) {
                dst[4 * i] = a[i].x, dst[4 * i + 1] = a[i].y, dst[4 * i + 2] = a[i].z, dst[4 * i + 3] = a[i].w;
            }
    };
    put4(P.gw_col, size_t(P.n_gwcol), gw_col);
    put4(P.gw_upd, size_t(sizes[4]), gw_upd);
    put4(P.gv_info, P.gv_info.size(), gv_info);
    if (gm_ptr && cap >= (long long)P.gm_ptr.size()) std::copy(P.gm_ptr.begin(), P.gm_ptr.end(), gm_ptr);
    if (gm_term && cap >= 2LL * sizes[5])
        for (int t = 0; t < sizes[5]; t++) {
            gm_term[2 * t] = P.gm_term[size_t(t)].x;
            gm_term[2 * t + 1] = P.gm_term[size_t(t)].y;
        }
    return 0;
}

// Test hook of the substitution sweeps' give-up path (needs a GPU): one
// solve of matrix `which` in place on rhs_dev (n doubles, local order) with
// instance 0 of its last factor of precision `prec`, in which the producer
// issues no piece from index stall_at of a sweep on (-1: off) or the
// consumers never release the stage of piece hold_at (-1: off), every wait
// bounded by `spin` polls.  *status_host receives PF_OK when the solve
// completed or PF_ERR_TIMEOUT when it gave up.  Synchronous.  Returns 0, or
// -1 for a bad argument, a matrix not factorised in that precision or a
// vector that does not fit shared memory, -2 when a CUDA call failed.
int gbpf_selftest_sweep(pf_ctx *ctx, int which, int prec, int stall_at, int hold_at, unsigned spin,
                        double *rhs_dev, int *status_host) {
    if (!ctx || which < 0 || which > 1 || (prec != PF_FP64 && prec != PF_FP32) || !rhs_dev ||
        !status_host || spin == 0)
        return -1;
    if (!ctx->ws.factored[which][prec]) return -1;
    const void *F = prec == PF_FP64 ? (const void *)ctx->ws.F64[which] : (const void *)ctx->ws.F32[which];
    int *st = ctx->ws.cstatus;
    cudaError_t e = launch_selftest_sweep(ctx->dm[which], prec, F, ctx->ws.TV[which][prec], rhs_dev, stall_at,
                                          hold_at, spin, st, ctx->smem_optin, nullptr);
    if (e == cudaErrorInvalidValue) return -1;
    if (e == cudaSuccess) e = cudaMemcpy(status_host, st, sizeof(int), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? 0 : -2;
}

// Test hook (host only, no GPU needed): the warp tasks of the tail factor
// of matrix `which` and the position of every target in its level.
// *ntask receives the number of tasks; tasks (4 ints each) and tipos (ng
// ints) are copied when cap covers them.  Returns 0, or -1 for a bad argument
// or a matrix that has not been analysed.
int gbpf_debug_tail_tasks(const pf_ctx *ctx, int which, int *ntask, int *tasks, int *tipos, int cap) {
    if (!ctx || !ntask || which < 0 || which > 1) return -1;
    const gbpf::HostMat &H = ctx->hm[which];
    if (H.lvl_ptr.empty()) return -1;
    *ntask = int(H.ttask.size());
    if (tasks && cap >= 4 * int(H.ttask.size()))
        for (size_t i = 0; i < H.ttask.size(); i++) {
            tasks[4 * i] = H.ttask[i].x;
            tasks[4 * i + 1] = H.ttask[i].y;
            tasks[4 * i + 2] = H.ttask[i].z;
            tasks[4 * i + 3] = H.ttask[i].w;
        }
    if (tipos && cap >= H.ft_ng) std::copy(H.tipos.begin(), H.tipos.begin() + H.ft_ng, tipos);
    return 0;
}

// Test hook (host only, no GPU needed): the partitioned inverse of the
// narrow top of matrix `which` (tail form 3).  sizes[10] receives {n, t0, nt,
// forward chunks, backward chunks, forward entries, backward entries, pieces
// of pf3, pieces of pb3, entries of L_TT}; when cap (ints per array) covers
// them, par (nt), fr and br (nt + 1), fc and bc (2 per chunk), fj, fs, bj,
// bs and bd (one per entry) are copied.  Returns 0, or -1 for a bad argument
// or a matrix that has not been analysed.
int gbpf_debug_tail_inverse(const pf_ctx *ctx, int which, int *sizes, int *par, int *fr, int *fc, int *fj,
                            int *fs, int *br, int *bc, int *bj, int *bs, int *bd, int cap) {
    if (!ctx || !sizes || which < 0 || which > 1) return -1;
    const gbpf::HostMat &H = ctx->hm[which];
    if (H.lvl_ptr.empty()) return -1;
    const bool on = !H.pf3.empty() && H.tw_ne > 0;
    const int nfc = on ? int(H.twfr.back()) : 0, nbc = on ? int(H.twbr.back()) : 0;
    sizes[0] = H.n;
    sizes[1] = H.t0;
    sizes[2] = on ? H.nt : 0;
    sizes[3] = nfc;
    sizes[4] = nbc;
    sizes[5] = on ? H.tw_nfe : 0;
    sizes[6] = on ? H.tw_nbe : 0;
    sizes[7] = int(H.pf3.size());
    sizes[8] = int(H.pb3.size());
    sizes[9] = on ? H.tw_ne : 0;
    if (!on) return 0;
    auto put = [&](const std::vector<int> &v, int count, int *dst) {
        if (dst && cap >= count) std::copy(v.begin(), v.begin() + count, dst);
    };
    auto put2 = [&](const std::vector<int2> &v, int count, int *dst) {
        if (dst && cap >= 2 * count)
            for (int k = 0; k < count; k++) {
                dst[2 * k] = v[size_t(k)].x;
                dst[2 * k + 1] = v[size_t(k)].y;
            }
    };
    put(H.twpar, H.nt, par);
    put(H.twfr, H.nt + 1, fr);
    put(H.twbr, H.nt + 1, br);
    put2(H.twfc, nfc, fc);
    put2(H.twbc, nbc, bc);
    put(H.twfj, H.tw_nfe, fj);
    put(H.twfs, H.tw_nfe, fs);
    put(H.twbj, H.tw_nbe, bj);
    put(H.twbs, H.tw_nbe, bs);
    put(H.twbd, H.tw_nbe, bd);
    return 0;
}

// Test hook (host only, no GPU needed): the CSR copy of L's pattern and its
// maps to the CSC one, and the off-diagonal pattern of A used by residuals,
// of matrix `which`.  sizes[4] receives {n, nnz, offLc, entries of A's
// pattern}; Fp (n + 1), Fc, Fpos, Cpos (nnz each), Ap (n + 1), Aj and Apos
// are copied when cap (ints per array) covers them.  Returns 0, or -1 for a
// bad argument or a matrix that has not been analysed.
int gbpf_debug_csr(const pf_ctx *ctx, int which, int *sizes, int *Fp, int *Fc, int *Fpos, int *Cpos,
                   int *Ap, int *Aj, int *Apos, int cap) {
    if (!ctx || !sizes || which < 0 || which > 1) return -1;
    const gbpf::HostMat &H = ctx->hm[which];
    if (H.lvl_ptr.empty() || H.Cp.empty()) return -1;
    const int nnz = H.Cp.back(), na = int(H.Aj.size());
    sizes[0] = H.n;
    sizes[1] = nnz;
    sizes[2] = H.offLc;
    sizes[3] = na;
    auto put = [&](const std::vector<int> &v, int count, int *dst) {
        if (dst && cap >= count) std::copy(v.begin(), v.begin() + count, dst);
    };
    put(H.Fp, H.n + 1, Fp);
    put(H.Fc, nnz, Fc);
    put(H.Fpos, nnz, Fpos);
    put(H.Cpos, nnz, Cpos);
    put(H.Ap, H.n + 1, Ap);
    put(H.Aj, na, Aj);
    put(H.Apos, na, Apos);
    return 0;
}

}  // extern "C"
