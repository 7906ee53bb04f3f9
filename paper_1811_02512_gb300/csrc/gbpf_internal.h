// gbpf_internal.h -- structures shared by the host analysis (gbpf_host.cpp)
// and the device kernels (gbpf_kernels.cu) of libgbpf.  Not part of the ABI.
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "gbpf.h"

namespace gbpf {

// Payload budget of one staged piece of a substitution sweep (bytes): the
// row pointers, column indices and values of a run of rows (columns) of one
// level, copied into shared memory by one TMA bulk transfer group.
constexpr int kPieceBytes = 8192;
constexpr int kPieceSlack = 128;
constexpr int kRingStages = 4;  // stages of the staging ring (one piece each)

// One staged piece: rows (columns) [r0, r1) whose entries are [e0, e1) of
// the CSR (CSC) arrays, all in level order.  mode: 0 one thread per row,
// 1 groups of 8 lanes per row (whole block), 2 warp 0 alone over rows of the narrow
// levels l0..l1, 3 warp 0 alone over part [e0, e1) of the single row r0 (a
// row too long for one stage); run_end: for modes 2, 3 and 4, the first
// piece after the run of single-warp pieces.  Mode 0/1/3 pieces lie in one
// level.  The sweeps with a scatter tail add: 4 warp 0 alone over the slot
// rows [e0/32, e1/32) of the tail levels r0..r1-1 of a scatter schedule
// (l0 = first tail row); 5 groups of 4 lanes per row over the entries of the tail
// rows in columns below the tail; 6 one thread per row, inverse diagonal
// only.
struct Piece {
    int r0, r1, e0, e1;
    int mode, run_end, l0, l1;
};
constexpr int kSweepWarps = 16;   // warps of the blocks that run the sweeps
constexpr int kNarrowRows = 16;   // levels with at most this many rows run on one warp

// Device layout of one factorised matrix (B' or B'').  All indices are in
// "level order": the elimination steps sorted by (level, step), so every
// level of the elimination tree is a contiguous range and the strict lower
// factor L stays lower triangular (a parent is always on a higher level).
// Per-instance factor values: [D: n | Dinv: 1/D | Lc: L by column (CSC) |
// Lr: L by row (CSR)], regions starting at multiples of 32 elements.
struct DevMat {
    int n = 0;           // dimension (buses in the matrix)
    int nnz = 0;         // strict-lower nonzeros of L
    int nlev = 0;        // levels of the elimination tree
    int max_col = 0;     // largest column count of L
    int64_t nupd = 0;    // scalar updates of one factorisation
    int offDi = 0, offLc = 0, offLr = 0, stride = 0;
    int npf = 0, npb = 0; // pieces of the forward / backward sweep
    int *bus = nullptr;        // [n]   level-order index -> global bus
    int *local = nullptr;      // [n]   level-order index -> local index
    int *new_of_bus = nullptr; // [nbus] global bus -> level-order index, -1 if absent
    int *lvl_ptr = nullptr;    // [nlev+1] level ranges
    int *Cp = nullptr, *Cr = nullptr;    // CSC of L: [n+1], [nnz] rows ascending
    int *Fp = nullptr, *Fc = nullptr;    // CSR of L: [n+1], [nnz] columns ascending
    int *Fpos = nullptr;       // [nnz] CSR entry -> CSC position
    int *uoff = nullptr;       // [nnz+1] CSR entry (c, k) -> start of its update map
    int *umap = nullptr;       // [nupd] target in column c: 0 diagonal, 1 + t = t-th entry
    // gather form of the same updates: target g = Cp[c] + c + t of column c
    // (t = 0 diagonal, 1 + t the t-th entry) receives sum over its list
    // gl[gp[g] .. gp[g+1]) of L[x] * L[y] * D[z] (x, y CSC positions, z column)
    int *gp = nullptr;         // [n + nnz + 1]
    int4 *gl = nullptr;        // [nupd] {x: L(i,k), y: L(c,k), z: k, w: 0}
    int *Cpos = nullptr;       // [nnz] CSC position -> CSR position
    int *src = nullptr;        // [n + nnz] Ybus position of every D and Lc slot, -1 = fill
    int *br_slot = nullptr;    // [3 nbranch] value slots (D f, D t, Lc (f,t)) or -1
    Piece *pf = nullptr, *pb = nullptr;  // forward (levels ascending), backward (descending)
    // Scatter tail: rows [t0, n) are the longest run of narrow levels at the
    // top of the elimination tree.  Their substitution runs on one warp as a
    // right-looking scatter: once x_j is final, x_i -= l x_j is applied to
    // every tail row i it reaches, each row owned by lane (i - t0) mod 32,
    // from a schedule of 32-slot rows per level.  SK: slot-row offsets per
    // tail level in sweep order; SI: (i - t0) | (j - t0) << 16 per slot, -1
    // empty; a lane's slots of one level are sorted by row.  The values of the slots (forward: L by column,
    // backward: L by row) and of the tail rows' entries in columns below t0
    // (PPp/PPc, by row) are gathered per instance after each factorisation
    // into [tv_f: forward slots | tv_b: backward slots | tv_p: entries below
    // t0] from the value slots TVsrc (-1: zero).
    int t0 = 0, nt = 0, ntl = 0;
    int npf2 = 0, npb2 = 0;
    Piece *pf2 = nullptr, *pb2 = nullptr;
    int *SKf = nullptr, *SIf = nullptr, *SKb = nullptr, *SIb = nullptr;
    int *PPp = nullptr, *PPc = nullptr, *ZP = nullptr;
    int tv_f = 0, tv_b = 0, tv_p = 0, tv_stride = 0;
    int *TVsrc = nullptr;
    // Tail factor: the columns [t0, n) factorised by one block in shared
    // memory, level by level.  Its gather targets are g0 + [0, ng) (g0 =
    // Cp[t0] + t0), its L entries Lc[e0 + [0, ne)) (e0 = Cp[t0]); per target
    // the A-value slot (tapos) and the first of its gather terms whose column
    // k is in the tail (gsplit; earlier terms have k < t0).
    int ft_ng = 0, ft_ne = 0, ft_g0 = 0, ft_e0 = 0;
    int *tapos = nullptr, *gsplit = nullptr;
    // the tail terms alone, packed {(x - e0) | (y - e0) << 16, k - t0}, by
    // target; ft_tmax = most terms of one tail level
    int2 *tterm = nullptr;
    int ft_tmax = 0;
    int ft_tterms = 0;         // tail terms in tterm
    // per tail level li: tlev[2 li] = {first target, end target, first term,
    // end term}, tlev[2 li + 1] = {first column - t0, end column - t0, first
    // task, end task}; the level's targets are reordered (position p of level
    // li holds target k with tipos[k] = first target + p);
    // per position: tinfo = {first term, end term (both relative to its
    // level's first), L entry - e0 (-1 for the diagonal), column - t0};
    // per task (a warp's work): ttask = {first position relative to the
    // level, targets, lanes per target G, 0}, 32 / G targets at most;
    // ft_kmax = most targets of one tail level
    int4 *tlev = nullptr, *tinfo = nullptr, *ttask = nullptr;
    int *tipos = nullptr;
    int ft_kmax = 0;
    int ft_ntask = 0;          // entries of ttask
    // Partitioned inverse of the same narrow top (tail form 3): with W =
    // L_TT^-1 of rows T = [t0, n) (unit lower; W(i, j) != 0 only for i an
    // ancestor of j), the sweeps run below the top (pf3: the wide levels and
    // the top rows' entries below t0, which leave c_T = b_T - L_TB z_B in
    // x[t0..n); pb3: the wide levels backward) and the top is two gathers,
    //   z_T = W c_T,   x_T = W^T D_T^-1 z_T,
    // each split into chunks of a few entries (twfc/twbc {first, end entry},
    // rows' chunk ranges twfr/twbr, entries' columns twfj/twbj - t0) whose
    // partial sums are added per row in chunk order.  Values per instance
    // (TW): [forward W(i, j) | backward W(j, i) / D(j)] at tw_boff, gathered
    // after each factorisation from the dense W (twfs/twbs: row * nt + col;
    // twbd: the D index of a backward entry).  The inverse itself is formed
    // by k_tail_inverse from the columns of L_TT (twcp, twcdep, twcpos, the
    // depth twdep and parent twpar of every top row).
    int npf3 = 0, npb3 = 0;
    Piece *pf3 = nullptr, *pb3 = nullptr;
    int tw_nfc = 0, tw_nbc = 0, tw_nfe = 0, tw_nbe = 0, tw_boff = 0, tw_stride = 0;
    int2 *twfc = nullptr, *twbc = nullptr;
    int *twfr = nullptr, *twbr = nullptr, *twfj = nullptr, *twbj = nullptr;
    int *twfs = nullptr, *twbs = nullptr, *twbd = nullptr;
    int *twpar = nullptr, *twcp = nullptr, *twcdep = nullptr, *twcpos = nullptr, *twdep = nullptr;
    int tw_ne = 0, tw_depmax = 0;
    int *Ap = nullptr, *Aj = nullptr, *Apos = nullptr;  // off-diagonal A (no fill), by row:
                                                       // column and value slot of each entry
    // Newton-Raphson Jacobian (2 x 2 blocks on the same pattern, B' only)
    int npfJ = 0, npbJ = 0;
    Piece *pfJ = nullptr, *pbJ = nullptr;
    int *srcT = nullptr;       // [nnz] Ybus position of the transposed entry (c, r) of each slot
    int jD = 0, jDi = 0, jLc = 0, jUc = 0, jLr = 0, jUr = 0, jstride = 0;  // block layout (elements)
};

// Cluster-distributed substitution program of one matrix for the
// single-case engine of gbpf_cluster.cu.  Every row of L (level order) has an
// owner CTA among kClCtas; a CTA's shared memory holds a "vector region" of
// words: its rows' entries of the solution (xb), and for its tail rows the
// forward intermediate c (tc) and the backward result (tx).  A reference to a
// word is owner << 16 | word.  The program of a CTA is a list of steps (one
// per level of the elimination tree, three for the tail), each a range of
// tasks {out word, in word, diagonal value index or -1, first entry}; a task
// computes X[out] = (diag ? val[diag] X[in] : X[in]) - sum over its entries
// of val[e] X(ref[e]).  Values are packed per CTA ([entries | diagonal
// values]) and gathered after every factorisation from vsrc {kind, a, b}:
// 0 the factor value F[a], 1 -W[a], 2 -W[a] F[b], W being the dense inverse
// of the tail block of L, row-major (W(it, jt) at W[it * nt + jt]); 3
// -GV[a], 4 -GV[a] F[b], 5 GV[a], GV the values of the grouped subtree steps.
constexpr int kClCtas = 16;
constexpr int kClGroupMax = 8;     // subtree levels per grouped step (at most)
constexpr int kClGroupDefault = 3; // subtree levels per step unless the tuning names another
constexpr int kClTailMax = 2048;   // largest tail whose dense inverse is formed
// T columns (one per warp) per block of k_tail_inverse: one warp per SM
// sub-partition, so that no two warps' chains of FP64 instructions share an
// FP64 unit
constexpr int kTailInvWarps = 4;
// shared memory of k_tail_inverse for a tail of nt rows with ne entries and
// paths of at most depth_max nodes (a tail whose need exceeds kTailInvSmem
// gets no inverse)
size_t tail_inverse_smem(int nt, int ne, int depth_max);
constexpr size_t kTailInvSmem = 160 * 1024;
struct ClMat {
    int nt = 0;                    // rows of the top set T with an inverse (0: none)
    int *tpar = nullptr;           // [nt] T-relative parent, -1 at a root
    int *tcp = nullptr;            // [nt + 1] columns of L_TT (all of a T column's rows are in T)
    int *tcdep = nullptr;          // [ntail_e] depth of each entry's row
    int *tcpos = nullptr;          // [ntail_e] factor position of each entry
    int ntail_e = 0;
    int *tdepth = nullptr;         // [nt] distance from its root
    int tdepth_max = 0;            // longest path in T (nodes)
    int nval = 0;
    int4 *vsrc = nullptr;          // [nval] value sources
    double *vals = nullptr;        // [nval] gathered values
    int4 *tasks = nullptr;         // all CTAs' tasks, each CTA's ending in a sentinel
    int *tptr = nullptr;           // [C + 1]
    int4 *steps = nullptr;         // all CTAs' steps {first task, end task, lanes per task,
                                   // 1: a cluster barrier follows (0: the CTA's own)}, CTA-relative
    int *sptr = nullptr;           // [C + 1]
    int *refs = nullptr, *eptr = nullptr;  // entry references, [C + 1]
    int *vptr = nullptr;           // [C + 1] value blocks
    int *rhsref = nullptr;         // [nbus] word of the bus's right-hand side, -1: not in the matrix
    int *xref = nullptr;           // [nbus] word of the bus's solution, -1: not in the matrix
    // byte offsets of the CTA's regions in dynamic shared memory
    int so_x = 0, so_tasks = 0, so_steps = 0, so_addr = 0, so_vals = 0;
    // Grouped subtree steps: with `group` g > 1 the subtree levels run g at a
    // time, each group through the inverse W_G of its block of L (unit lower,
    // W(i, j) != 0 only for j a descendant of i within the group):
    //   forward  z_i = b_i + sum_{j desc} W(i,j) b_j - sum_k M(i,k) z_k,
    //            M(i,k) = sum_{j in {i} + desc} W(i,j) L(j,k), k below the group;
    //   backward x_i = z_i / d_i + sum_{j anc} W(j,i) z_j / d_j - sum_k M'(i,k) x_k,
    //            M'(i,k) = sum_{j in {i} + anc} W(j,i) L(k,j), k above the group.
    // The group values GV = [W entries | combined entries] are formed after
    // every factorisation: gw_col per inverse column j {first update, end
    // update, GV index of W(path[1], j), path length P}, gw_upd {p, q, factor
    // position of L(path[q], path[p]), 0} (w_q -= L w_p along the path);
    // gm_ptr / gm_term per combined entry its terms {W index or -1 for the
    // identity, factor position of the L entry}, summed in order.
    int n_gwcol = 0, n_gw = 0, n_gm = 0;
    int4 *gw_col = nullptr, *gw_upd = nullptr;
    int *gm_ptr = nullptr;
    int2 *gm_term = nullptr;
    double *gv = nullptr;          // [n_gw + n_gm]
};

// Host form of a ClMat.
struct HostCl {
    int ok = 0;                    // the program fits (top set small enough for its inverse)
    int nt = 0, nx = 0, tdepth_max = 0;
    int group = 1;                 // subtree levels per step (see ClMat)
    // values of the grouped steps (see ClMat): inverse columns, their updates,
    // the combined entries' terms, and what every value is (for tests:
    // {0, row, column} an entry of a group's inverse, {1, row, k} a forward
    // combined entry, {2, row, k} a backward one)
    std::vector<int4> gw_col, gw_upd, gv_info;
    std::vector<int> gm_ptr;
    std::vector<int2> gm_term;
    int n_gwcol = 0, n_gw = 0, n_gm = 0;
    std::vector<int> tnode;        // level-order rows of the top set, ascending
    std::vector<int> tpar, tcp, tcdep, tcpos, tdepth;
    std::vector<int4> vsrc, tasks, steps;
    std::vector<int> tptr, refs, eptr, vptr, sptr, rhsref, xref;
    size_t max_tasks = 0, max_steps = 0, max_e = 0, max_v = 0;  // per CTA (tasks with the sentinel)
    int64_t bottom_load_max = 0, bottom_load_avg = 0;          // subtree weight per CTA
};

// Host copy of the symbolic data of one matrix.  Step numbering (the
// minimum-degree elimination order) for the published symbolic result;
// level order for the device layout.
struct HostMat {
    int n = 0;
    std::vector<int> bus;      // local -> global bus (ascending)
    std::vector<int> perm;     // step -> local
    std::vector<int> iperm;    // local -> step
    std::vector<int64_t> Lp;
    std::vector<int> Li;
    std::vector<int> parent, level;
    int nlev = 0;
    int max_col = 0;
    int64_t nupd = 0;
    // device layout (level order)
    std::vector<int> neword;       // level order -> step
    std::vector<int> new_of_step;  // step -> level order
    std::vector<int> bus_new, local_new, new_of_bus;
    std::vector<int> lvl_ptr;
    std::vector<int> Cp, Cr, Fp, Fc, Fpos, uoff, umap, src, br_slot, gp, Cpos;
    std::vector<int4> gl;
    std::vector<int> csc_of_steppos;  // step-numbered CSC position -> level-order CSC position
    std::vector<int> Ap, Aj, Apos;    // off-diagonal pattern of A by row (both triangles, no fill)
    std::vector<Piece> pfJ, pbJ;
    std::vector<int> srcT;
    int jD = 0, jDi = 0, jLc = 0, jUc = 0, jLr = 0, jUr = 0, jstride = 0;
    std::vector<Piece> pf, pb;
    int offDi = 0, offLc = 0, offLr = 0, stride = 0;
    int t0 = 0, nt = 0, ntl = 0;
    std::vector<Piece> pf2, pb2;
    std::vector<int> SKf, SIf, SKb, SIb, PPp, PPc, TVsrc;
    int tv_f = 0, tv_b = 0, tv_p = 0, tv_stride = 0;
    int ft_ng = 0, ft_ne = 0, ft_g0 = 0, ft_e0 = 0;
    std::vector<int> tapos, tcol, gsplit, tptr;
    std::vector<int2> tterm;
    int ft_tmax = 0;
    std::vector<int4> tlev, tinfo, ttask;
    std::vector<int> tipos;
    int ft_kmax = 0;
    // partitioned inverse of the narrow top (see DevMat)
    std::vector<Piece> pf3, pb3;
    std::vector<int> twpar, twcp, twcdep, twcpos, twdep;
    int tw_ne = 0, tw_depmax = 0;
    std::vector<int> twfr, twbr, twfj, twbj, twfs, twbs, twbd;
    std::vector<int2> twfc, twbc;
    int tw_nfe = 0, tw_nbe = 0, tw_boff = 0, tw_stride = 0;
};

// Device arrays of the network and of the case batch.
struct DevNet {
    int nbus = 0, nbr = 0, nnz = 0;
    // network tables
    int *btype = nullptr;
    double *pd = nullptr, *qd = nullptr, *gs = nullptr, *bs = nullptr, *pg = nullptr;
    double *vset = nullptr, *va0 = nullptr;
    int *bf = nullptr, *bt = nullptr, *bstatus = nullptr;
    double *br = nullptr, *bx = nullptr, *bb = nullptr, *btap = nullptr;
    // Ybus pattern (CSR, ascending columns) and base values
    int *rowptr = nullptr, *col = nullptr, *ydiag = nullptr;
    double *G = nullptr, *B = nullptr, *Bp = nullptr;  // Bp: XB B' on the Ybus pattern
    // bus incidence: for bus i, entries inc_ptr[i]..: branch, side (0 from, 1 to), off-diag position
    int *inc_ptr = nullptr, *inc_br = nullptr, *inc_side = nullptr, *inc_pos = nullptr;
    int *br_pos = nullptr;   // [nbr*4] Ybus positions (ff, tt, ft, tf)
    // off-diagonal Ybus entries: {position, first, end, 0} into yoff_br, the
    // branches whose pi model reaches the entry (ascending branch index)
    int noff = 0;
    int4 *yoff = nullptr;
    int *yoff_br = nullptr;
    // Thread order of the nodal mismatch: the buses by Ybus row length
    // (stable), within windows of 1,024 buses (mis_ord, one CTA per case)
    // and within each of the kClCtas slices of the cluster engine
    // (mis_ord_cl).  An
    // FP64 instruction costs a GB300 SM sub-partition the same whatever
    // number of its warp's lanes is active, so a warp's rows should be of
    // one length.
    int *mis_ord = nullptr, *mis_ord_cl = nullptr;
};

struct DevCases {
    int ncase = 0;
    int ninst = 1;            // factor instances: 0 = base, 1.. = outage cases
    int *outage = nullptr;    // [ncase] branch or -1
    int *inst = nullptr;      // [ncase] factor instance of each case
    int *inst_outage = nullptr; // [ninst] branch of each instance (-1 for base)
    double *Psp = nullptr, *Qsp = nullptr; // [ncase][nbus]
};

// Cases in lane groups of 32 for the lockstep batched engine (gbpf_batch.cu).
// State arrays are [bus][ncp] (lane fastest), solve vectors [group][nbus][32].
struct LaneSet {
    int ngroups = 0, ncp = 0, nown = 0;
    int *gcase = nullptr;    // [ncp] case of each lane, -1 = empty lane
    int *ginst = nullptr;    // [ncp] factor instance of each lane (0 for empty lanes)
    int *gshared = nullptr;  // [ngroups] 1: all lanes use instance 0
    int *gown = nullptr;     // [ngroups] index among own-factor groups, -1 if shared
    int *owngroup = nullptr; // [nown] group of each own-factor group
    double *vm = nullptr, *va = nullptr, *cs = nullptr, *sn = nullptr, *iv = nullptr;
    double *e = nullptr, *f = nullptr, *psp = nullptr, *qsp = nullptr;  // [nbus][ncp]
    double *maxmis = nullptr, *lastmis = nullptr;                       // [ncp]
    int *active = nullptr, *status = nullptr, *iters = nullptr, *irs = nullptr;  // [ncp]
    int *nactive = nullptr;
    void *X = nullptr;       // [ngroups][nbus][32] in the solve precision
    double *b = nullptr, *x64 = nullptr;  // [ngroups][nbus][32]
    void *LF0 = nullptr, *LF1 = nullptr;  // [nown][stride][32] interleaved own factors
    int prec = -1;
};

struct FactorJob;

struct Workspace {
    // factor storage per matrix and precision: [ninst][stride]
    double *A[2] = {nullptr, nullptr};       // assembled values (FP64), per instance
    double *F64[2] = {nullptr, nullptr};
    float *F32[2] = {nullptr, nullptr};
    int *fstatus[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}}; // [mat][prec] per instance
    bool factored[2][2] = {{false, false}, {false, false}};
    int ninst_alloc = 0;
    // dependency-driven factor: per matrix, column-done flags [ninst][n]
    // (a column is done when its flag equals the epoch of the current
    // factorisation), the column counter and abort flag, diagonal maxima
    unsigned *fdone[2] = {nullptr, nullptr};
    unsigned *fsync[2] = {nullptr, nullptr};  // [0] next column, [1] abort
    double *famax[2] = {nullptr, nullptr};    // [ninst]
    unsigned fepoch[2] = {0u, 0u};
    void *TV[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [mat][prec] tail values
    void *TP[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [mat][prec] tail targets' parts
    void *TW[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [mat][prec] tail inverse values (instance 0)
    double *TWd[2] = {nullptr, nullptr};  // [mat] dense inverse of the narrow top (FP64, nt x nt)
    // low-rank outages, per matrix: Z [ninst][2][n] of the factor type (per
    // precision), K [ninst][4], solve scratch
    void *LZ[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    double *LK[2] = {nullptr, nullptr};
    void *Lscr[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    // second stream for the B'' factorisation beside B' (fork/join events)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // per-case scratch
    double *ef = nullptr;     // [ncase][4*nbus] e, f, cos(theta), sin(theta)
    double *vec = nullptr;    // [ncase][3*nbus] rhs, refined FP64 solution, FP32 work vector
    double *bmax = nullptr;   // [ncase][16] per-CTA mismatch maxima and solve flag
    double *iv = nullptr;     // [ncase][nbus] 1 / V
    int *cstatus = nullptr;   // [ncase] run status
    pf_case_result *res = nullptr; // [ncase]
    int ncase_alloc = 0;
    double *lsbuf = nullptr;  // [ncase][nbus] load scales of the batch (kept for a cheap re-set)
    int *lsflag = nullptr;    // set when new load scales of the same cases are not all finite
    std::vector<int> case_out;  // host copy of the batch's outages (-1: none)
    // Newton-Raphson workspace (allocated on first use): block factors per
    // precision, the FP64 Jacobian and per-case factor status, [ncase][jstride]
    void *JF[2] = {nullptr, nullptr};
    double *JA = nullptr;
    int *jfstat[2] = {nullptr, nullptr};
    bool jfactored[2] = {false, false};
    double *xg6 = nullptr;    // [ncase][6*nbus] Newton right-hand side, refined x, FP32 work
    unsigned *jdone = nullptr;   // [ncase][n] Jacobian column done flags (epochs)
    unsigned *jsync = nullptr;   // [ncase][2]
    unsigned jepoch = 0;         // last epoch handed to a launch
    LaneSet lanes;
};

}  // namespace gbpf

namespace gbpf {
struct KernelStat {
    int64_t launches = 0;
    double ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};
}  // namespace gbpf

struct pf_ctx {
    int nbus = 0, nbr = 0;
    bool profiling = false;
    gbpf::KernelStat kstat[PF_K_COUNT];
    std::vector<pf_bus> bus;
    std::vector<pf_branch> branch;
    int slack = -1;
    // Ybus pattern (host)
    std::vector<int> rowptr, col;
    bool analyzed = false;
    gbpf::HostMat hm[2];
    gbpf::DevMat dm[2];
    gbpf::DevNet dn;
    gbpf::DevCases dc;
    gbpf::Workspace ws;
    bool on_device = false;   // network and symbolic data uploaded
    std::vector<int> ydiag, inc_ptr, inc_br, inc_side, inc_pos, br_pos, yoff_br;
    std::vector<int4> yoff;
    std::vector<int> mis_ord, mis_ord_cl;
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    size_t smem_per_sm = 0;
    std::string err;
    std::vector<void *> allocations;  // everything owned by the context
    pf_tuning tune = {0, 0, 0, 0, 0, 0, 0.0};  // kernel mappings (pf_autotune / pf_set_tuning)
    // programs of the cluster engine (host, device), their tail-inverse
    // scratch and the dynamic shared memory of one CTA
    gbpf::HostCl hcl[2];
    gbpf::ClMat cl[2];
    double *clW[2] = {nullptr, nullptr};
    size_t cl_smem = 0;
    int cl_group = gbpf::kClGroupDefault;  // subtree levels per step of the cluster engine's programs
    int tail_cl_max[2][2] = {{-1, -1}, {-1, -1}};  // [mat][prec] resident tail-factor clusters (-1: not asked)
    // CUDA graph of the device work of one fast decoupled pf_run_to_tol
    // (block and cluster engines), captured on an internal stream for a given
    // set of arguments (key) and replayed on the caller's stream; the launch
    // counts of one replay per kernel kind
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> gkey, gkey_last;
    int64_t glaunches[PF_K_COUNT] = {};
    bool graph_capturing = false;
    bool graphs_off = false;
    int set_gen = 0;  // bumped by every pf_set_cases (the batch's arrays are new)
};

namespace gbpf {

// Launch wrappers implemented in gbpf_kernels.cu.  All return cudaError_t of
// the launch (asynchronous errors surface at the next synchronising call).
cudaError_t launch_ybus(const DevNet &dn, cudaStream_t s);
cudaError_t launch_case_spec(const DevNet &dn, const DevCases &dc, const double *load_scale_dev,
                             cudaStream_t s, const int *skip = nullptr);
cudaError_t launch_finite_check(const double *x, long long n, int *bad, cudaStream_t s);
cudaError_t launch_assemble_slots(const DevNet &dn, const DevCases &dc, const DevMat &m, int which,
                                  double *A, cudaStream_t s, int ninst = -1);
cudaError_t launch_branch_flows(const DevNet &dn, const DevCases &dc, const double *vm, const double *va,
                                int ncase, double *flows, double *loss, cudaStream_t s);
struct FactorSync {
    unsigned *done = nullptr;  // [ninst][n]
    unsigned *sync = nullptr;  // [0] column counter, [1] abort flag
    double *amax = nullptr;    // [ninst]
    unsigned epoch = 0;
    unsigned spin = 0;
    int nsm = 0;
    int mode = 0;              // 0 auto, 1 dependency-driven, 2 block per instance
    int blocks_per_sm = 2;     // dependency-driven grid: blocks per SM
    bool tail = true;          // factor the narrow top in one block (k_factor_tail) when it fits
    size_t smem_optin = 0;
    void *partg = nullptr;     // [ninst][ft_ng] of the factor type: the tail targets' parts
                               // from columns below the tail (k_factor_tail_pre)
    bool tail_cluster = false; // the tail factor of every instance on a cluster of kTailCtas CTAs
};
constexpr int kTailCtas = 16;  // CTAs of the tail factor's cluster (one per SM)
size_t factor_tail_smem(const DevMat &m, int prec);
// Clusters of the tail factor that can be resident at once (0: none).
int factor_tail_clusters(const DevMat &m, int prec);
cudaError_t launch_factor(const DevMat &m, int prec, const double *A, void *F, int ninst,
                          int *fstatus, const FactorSync &fs, cudaStream_t s);
// Longest column (strict-lower entries) the dependency-driven factor takes.
constexpr int kDepMaxCol = 255;
// One matrix (single instance) of a packed factorisation.
struct FactorJob {
    DevMat m;
    const double *A;
    void *F;
    void *TV;
    int *fstatus;
    unsigned *done;
    double *amax;
    unsigned epoch;
};
// Factorises the matrices jobs_dev[0..njob) in one dependency-driven launch
// over the work items (job, column) of items_dev (every column after the
// columns it depends on), then gathers their tail values.  sync_dev: the
// column counter and abort flag.
cudaError_t launch_factor_jobs(const FactorJob *jobs_dev, int njob, const int2 *items_dev,
                               unsigned nitems, unsigned *sync_dev, int prec, int nsm, cudaStream_t s);
// Partitioned inverse of the narrow top of instance 0 (tail form 3): the
// dense W = L_TT^-1 into Wd (FP64) and the gathered values into TW (prec).
cudaError_t launch_tail_w(const DevMat &m, int prec, const void *F, double *Wd, void *TW, cudaStream_t s);
cudaError_t launch_tail_values(const DevMat &m, int prec, const void *F, void *TV, int ninst,
                               cudaStream_t s);
cudaError_t launch_solve(const DevMat &m, int prec, const void *F, const void *TV,
                         const int *inst_of_case, double *rhs, int ncase, void *gvec, int *status,
                         size_t smem_optin, cudaStream_t s);
// Self-test of the sweeps' give-up path (one block, instance 0 of F; the
// solve vector must fit shared memory): see k_selftest_sweep.
cudaError_t launch_selftest_sweep(const DevMat &m, int prec, const void *F, const void *TV, double *rhs,
                                  int stall_at, int hold_at, unsigned spin, int *status,
                                  size_t smem_optin, cudaStream_t s);
cudaError_t launch_mismatch(const DevNet &dn, const DevCases &dc, const double *vm, const double *va,
                            double *dp, double *dq, double *maxmis, double *ef, int ncase,
                            cudaStream_t s);
struct NrLaunch;
// fb (optional): the Newton-Raphson launch that unconverged cases fall back
// to inside the same launch (ignored when its factor scratch does not fit);
// TW0/TW1 (optional): tail-inverse values of instance 0 (tail form 3).
cudaError_t launch_fdpf(const DevNet &dn, const DevCases &dc, const DevMat *m, int prec,
                        const void *F0, const void *F1, const void *TV0, const void *TV1,
                        const double *A0, const double *A1,
                        const int *fstat0, const int *fstat1, const pf_run_opts &o, double *vm,
                        double *va, double *ef, double *iv, double *xg, double *bmax,
                        pf_case_result *res, size_t smem_optin, size_t smem_per_sm, int cluster,
                        int threads, cudaStream_t s,
                        const void *Z0 = nullptr, const void *Z1 = nullptr, const double *K0 = nullptr,
                        const double *K1 = nullptr, const NrLaunch *fb = nullptr,
                        const void *TW0 = nullptr, const void *TW1 = nullptr);
// Z = A^-1 U and K = (I - S U^T Z)^-1 S of every outage instance of matrix
// `which` from the base factor F (instance 0): the low-rank form of the
// outage cases.  gvec: [2 (ninst - 1)][n] scratch of the factor type.
cudaError_t launch_lowrank(const DevMat &m, const DevNet &dn, const DevCases &dc, int which, int prec,
                           const void *F, const void *TV, void *Z, double *Kd, void *gvec, int *status,
                           size_t smem_optin, cudaStream_t s);
int fdpf_cluster_size(int ncase, int num_sms, int prec, size_t smem_optin, int nmax);

// One grid of a pack (uneven multi-grid batch): its device network, case,
// layout, factors and per-case scratch, with vm/va inside the pack's
// concatenated state vectors and res inside the pack's result array.
struct PackGrid {
    DevNet dn;
    DevCases dc;
    DevMat m[2];
    const void *F0, *F1, *TV0, *TV1;
    const double *A0, *A1;
    const int *fs0, *fs1;
    double *vm, *va, *ef, *iv, *xg, *bmax;
    pf_case_result *res;
};
size_t run_args_bytes();
// Runs every grid of a pack to tolerance in one persistent launch (grids
// taken largest first, order_host); args_dev/order_dev/counter_dev are
// device scratch of ngrid run arguments, ngrid ints and one counter.
cudaError_t launch_pack(const PackGrid *grids, int ngrid, int prec, const pf_run_opts &o,
                        const int *order_host, void *args_dev, int *order_dev, unsigned *counter_dev,
                        size_t smem_optin, int nsm, cudaStream_t s);

// One launch of the Newton-Raphson kernel (adjoint = false) or of the
// adjoint kernel (adjoint = true).
struct NrLaunch {
    DevNet dn;
    DevCases dc;
    DevMat m;
    void *F = nullptr;
    double *A = nullptr;
    int *fstat = nullptr;
    pf_run_opts o{};
    int prec = PF_FP64;
    double *vm = nullptr, *va = nullptr, *ef = nullptr, *xg = nullptr, *bmax = nullptr;
    pf_case_result *res = nullptr;
    const double *gva = nullptr, *gvm = nullptr;
    double *dJdP = nullptr, *dJdQ = nullptr;
    size_t smem_optin = 0;
    int cluster = 1;
    bool adjoint = false;
    int factor_now = 0;
    unsigned *jdone = nullptr;  // [ncase][n] column done flags of the Jacobian factor
    unsigned *jsync = nullptr;  // [ncase][2] column counter, abort flag
    unsigned epoch0 = 0;        // factorisation k of this launch publishes epoch0 + k
};
cudaError_t launch_nr(const NrLaunch &L, cudaStream_t s);
int nr_cluster_size(const DevMat &m, int ncase, int num_sms, int prec, size_t smem_optin);
struct LaneRun {
    DevNet dn;
    DevCases dc;
    DevMat m0, m1;
    LaneSet L;
    const void *F0 = nullptr, *F1 = nullptr;
    const int *fs0 = nullptr, *fs1 = nullptr;
    const double *A0 = nullptr, *A1 = nullptr;
    pf_run_opts o{};
    int prec = PF_FP64;
    double *vm = nullptr, *va = nullptr;
    pf_case_result *res = nullptr;
    int use_graph = 1;
    size_t smem_optin = 0;
};
cudaError_t lane_run(const LaneRun &r, cudaStream_t s);
int lane_width(int nmax, int prec, size_t smem_optin);

// Single-case engine with the substitutions spread over a cluster
// (gbpf_cluster.cu): the top set's inverse of one matrix after its
// factorisation (W: nt^2 doubles of scratch, launched on that matrix's
// stream), the groups' inverses and packed values of both matrices once
// both inverses are done, and the iteration kernel (smem: dynamic shared
// memory of one CTA).
cudaError_t launch_cl_inverse(const ClMat &m, const double *F, double *W, cudaStream_t s);
cudaError_t launch_cl_prepare(const ClMat &m0, const ClMat &m1, const double *F0, const double *F1,
                              double *W0, double *W1, cudaStream_t s);
cudaError_t launch_fdpf_cl(const DevNet &dn, const DevCases &dc, const ClMat &m0, const ClMat &m1,
                           const int *fs0, const int *fs1, const pf_run_opts &o, double *vm, double *va,
                           double *ef, double *iv, double *bmax, pf_case_result *res, size_t smem,
                           cudaStream_t s, const NrLaunch *fb = nullptr, size_t smem_optin = 0);
bool fdpf_cl_fits(size_t smem);

cudaError_t launch_objective(const DevNet &dn, const DevCases &dc, const double *vm, const double *va,
                             double *ef, double *J, double *gva, double *gvm, cudaStream_t s);

}  // namespace gbpf
