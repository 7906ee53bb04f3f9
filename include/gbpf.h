/*
 * gbpf.h -- C ABI of the GB300 graph-based power-flow library (libgbpf.so).
 *
 * The library implements the hot path of Section III of "Graph Based Power
 * Flow Calculation for Energy Management System" (arxiv 1811.02512): nodal-
 * parallel formation of the bus admittance matrix (Section III.A, FormMatrixA)
 * and of the P/Q mismatch (Section II.A), hierarchical-parallel sparse LDU
 * factorisation over the levels of the elimination tree (Sections II.B and
 * III.B, Eqs. 1-3), and level-scheduled forward substitution, normalisation
 * (Eq. 4) and back substitution (Section III.C), driven by the fast-decoupled
 * and Newton-Raphson power-flow iterations (Section III).
 *
 * Conventions for every entry point:
 *  - All quantities are per unit; angles in radians.
 *  - Buses are numbered 0..nbus-1 in the order given to pf_create.  The
 *    unknowns of a matrix are its buses in ascending bus order ("local"
 *    order): B' and the Newton-Raphson Jacobian use every non-slack bus, B''
 *    every PQ bus.
 *  - Pointers named *_dev are device memory owned by the caller (for example
 *    torch.Tensor.data_ptr()); other pointers are host memory owned by the
 *    caller.  pf_create copies its inputs; the library never keeps a caller
 *    pointer beyond the call.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls marked
 *    "asynchronous" only enqueue work on it; the others return after their
 *    work is complete.
 *  - Batched vectors are case-major: element (c, i) of a [ncase][len] array
 *    is at c * len + i.
 *  - Every call returns a pf_status and never aborts, traps or exits; a
 *    failing call leaves a message for pf_last_error.  Device-side failures
 *    (singular pivot, non-finite value, exhausted wait) are reported per case
 *    through status words, never through a device trap.
 *  - A context is not thread safe; use one context per host thread.
 */
#ifndef GBPF_H
#define GBPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pf_ctx pf_ctx;

typedef enum {
    PF_OK = 0,
    PF_ERR_ARG = 1,           /* invalid argument or input table */
    PF_ERR_ISLAND = 2,        /* a bus is not connected to the slack bus */
    PF_ERR_SINGULAR = 3,      /* pivot |d_j| <= 1e-14 max |a_jj| during the factor */
    PF_ERR_NONFINITE = 4,     /* NaN or Inf reached a pivot, mismatch or state */
    PF_ERR_NOT_CONVERGED = 5, /* iteration limit reached above the tolerance */
    PF_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
    PF_ERR_CUDA = 7,          /* a CUDA runtime call failed */
    PF_ERR_OOM = 8,           /* host or device allocation failed */
    PF_ERR_STATE = 9          /* call out of order (e.g. pf_solve before pf_factor) */
} pf_status;

enum { PF_BUS_PQ = 1, PF_BUS_PV = 2, PF_BUS_SLACK = 3 };
enum { PF_MAT_BP = 0, PF_MAT_BPP = 1 }; /* B' (non-slack buses), B'' (PQ buses) */
enum { PF_FDPF = 1, PF_NR = 2 };
enum { PF_FP64 = 0, PF_FP32 = 1 };

/* One bus.  type: PF_BUS_PQ / PF_BUS_PV / PF_BUS_SLACK (exactly one slack).
 * Specified injection: P = pg - pd (non-slack), Q = -qd (PQ).  Shunt gs + j bs.
 * vset: voltage magnitude of PV and slack buses; va: slack angle. */
typedef struct {
    int32_t id, type;
    double pd, qd, gs, bs, pg, vset, va;
} pf_bus;

/* One branch (pi model).  Series r + jx, total line charging b (b/2 at each
 * end), off-nominal tap ratio on the from side (0 or 1 = none, no phase
 * shift), status 1 = in service, 0 = out (it keeps its matrix slot). */
typedef struct {
    int32_t from, to;
    double r, x, b, tap;
    int32_t status;
} pf_branch;

/* Sizes produced by pf_analyze, index [PF_MAT_BP] and [PF_MAT_BPP]. */
typedef struct {
    int32_t n[2];        /* matrix dimension (buses) */
    int64_t nnz_l[2];    /* strict-lower nonzeros of L (fill included) */
    int32_t nlevels[2];  /* levels of the elimination tree (leaves = 1) */
    int32_t max_col[2];  /* largest column count of L (diagonal excluded) */
    int64_t nupdates[2]; /* scalar update operations of one numeric factor */
    int32_t nnz_ybus;    /* nonzeros of the bus admittance pattern */
    double analyze_ms;   /* host wall time of the analysis */
} pf_symbolic_info;

/* Options of pf_run_to_tol. */
typedef struct {
    int32_t method;     /* PF_FDPF (XB fast decoupled) or PF_NR */
    int32_t precision;  /* PF_FP64, or PF_FP32 factor/substitution with FP64
                           mismatch, residual and refinement */
    double tol;         /* converged when max(|dP| non-slack, |dQ| PQ) <= tol */
    int32_t max_iter;   /* NR steps or FDPF half-iteration pairs */
    int32_t ir_max;     /* PF_FP32: refinement corrections per linear solve */
    double ir_tol;      /* PF_FP32: stop refining at ||r||inf <= ir_tol ||rhs||inf ... */
    double ir_abs;      /* ... or at ||r||inf <= ir_abs (0 = 0.01 tol: a linear-solve
                           residual that small cannot change a convergence decision) */
    int32_t flat_start; /* 1: theta = slack angle / 0, V = 1 (PQ) or vset; 0: use vm/va */
    int32_t spin_limit; /* bound on every device-side wait (0 = library default) */
    int32_t engine;     /* PF_ENGINE_AUTO, PF_ENGINE_BLOCK, PF_ENGINE_LANES or
                           PF_ENGINE_CLUSTER (FDPF only) */
    int32_t fallback;   /* FDPF only (Section III, FDPF first, then NR): 1 = a case
                           the fast decoupled iteration leaves unconverged
                           (PF_ERR_NOT_CONVERGED, PF_ERR_NONFINITE) switches to
                           Newton-Raphson from a flat start on the device, inside
                           the same iteration launch (at most 30 Newton steps,
                           same precision and tolerance; no host synchronisation,
                           converged cases are not re-run); its result then
                           reports method PF_NR.  The BLOCK and CLUSTER engines
                           carry it (a run that asks for it does not use LANES);
                           ignored where the Newton-Raphson factor scratch does
                           not fit shared memory (the grid's Newton-Raphson runs
                           would not launch either).  Allocates the Newton-Raphson
                           storage on first use. */
} pf_run_opts;

/* Engines of pf_run_to_tol.  BLOCK: one thread block (or, for a few large
 * cases, a 16-block cluster) per case, each case iterating independently in
 * one persistent launch.  LANES (FDPF only): the batch advances in lockstep
 * in groups of 32 cases, one case per lane; the mismatch, convergence test
 * and update run over (bus, case) pairs, each substitution over blocks of
 * 4, 2 or 1 cases whose vectors fit in shared memory, and one half-iteration
 * pair is a CUDA graph replayed until every case has retired.  CLUSTER
 * (FDPF, FP64, a batch of one case without outage): the case runs on a
 * 16-block cluster that shares the substitutions as well as the mismatch --
 * every row of L belongs to one block, which keeps its factor entries in
 * shared memory for the whole run; a level of the elimination tree is one
 * step of all blocks followed by a cluster barrier, and the narrow top of
 * the tree is solved with the explicit inverse of its block of L (three
 * steps in all); it needs the factors' programs to fit in shared memory.
 * AUTO picks BLOCK; LANES and CLUSTER fall back to BLOCK where they do not
 * apply. */
enum { PF_ENGINE_AUTO = 0, PF_ENGINE_BLOCK = 1, PF_ENGINE_LANES = 2, PF_ENGINE_CLUSTER = 3 };

/* Kernel mappings of a context, chosen by pf_autotune (or set directly with
 * pf_set_tuning; 0 in a field = the library's default choice):
 *   engine   PF_ENGINE_BLOCK, PF_ENGINE_LANES or PF_ENGINE_CLUSTER, used
 *            by FDPF runs whose options ask for PF_ENGINE_AUTO;
 *   cluster  thread blocks per case of a single-case FDPF run (1, 8, 16;
 *            capped at what fits the GPU); with engine PF_ENGINE_CLUSTER
 *            instead the subtree levels per step of its substitutions (1 to
 *            8, 0 = 3): g levels of a CTA's subtrees are solved in one step
 *            through the inverse of their block of L (formed after every
 *            factorisation), so the per-level barriers drop g-fold at the
 *            cost of the inverse's extra entries;
 *   factor   1: dependency-driven factor over all SMs, 2: one thread block
 *            per instance (level by level);
 *   tail     1: narrow top of the elimination tree substituted as a one-warp
 *            scatter, 2: level by level (warp per narrow level), 3: through
 *            the top's partitioned inverse W = L_TT^-1 (z_T = W c_T, x_T =
 *            W^T D_T^-1 z_T: two parallel gathers instead of a level chain;
 *            W formed after every factorisation; block engine runs whose
 *            solves all use the base factor: one instance, or low-rank
 *            outages -- other runs use form 1);
 *   outage   1: every single-branch outage case has its own B'/B'' factors,
 *            2: outage cases reuse the base factors with a low-rank
 *            (Woodbury) correction of each solve by the outaged branch's
 *            share (block engine; FP32 runs still refine against each
 *            case's exact matrix in FP64);
 *   threads  threads of each block of the block engine when it runs one
 *            block per case (512, 256 or 128): smaller blocks let more
 *            cases share an SM (2, 4 or 6 to 8), so that their latency-bound
 *            substitutions overlap one another's FP64 mismatch work; a
 *            block of 256 or 128 threads keeps its solve vector in global
 *            memory (L1/L2) when shared memory would otherwise limit the
 *            cases per SM.
 * ms is the time of one run of the chosen mapping as measured by
 * pf_autotune (0 when set directly). */
typedef struct {
    int32_t engine;
    int32_t cluster;
    int32_t factor;
    int32_t tail;
    int32_t outage;
    int32_t threads;
    double ms;
} pf_tuning;

/* Per-case outcome of pf_run_to_tol. */
typedef struct {
    int32_t status;      /* pf_status of this case */
    int32_t iters;       /* NR steps, or FDPF half-iterations */
    int32_t ir_steps;    /* refinement corrections taken (PF_FP32) */
    int32_t method;      /* method that produced the result: PF_FDPF or PF_NR */
    double max_mismatch; /* last max |mismatch| evaluated */
} pf_case_result;

/* Builds a context from bus and branch tables (copied).  Checks indices,
 * impedances (finite, x != 0 or r != 0), exactly one slack bus and
 * connectivity to the slack bus (PF_ERR_ISLAND).  Synchronous. */
pf_status pf_create(const pf_bus *bus, int32_t nbus, const pf_branch *branch, int32_t nbranch,
                    pf_ctx **out);

/* Host symbolic analysis of B' and B'' (the Newton-Raphson Jacobian reuses
 * B''s): exact minimum-degree ordering (ties to the smallest bus), fill
 * pattern of L (Section II.B.1), elimination tree (Section II.B.2), level
 * sets (Section II.B, Table I: leaves are level 1), the level schedules and
 * the update lists of the left-looking factor; uploads them to the current
 * device.  info may be NULL.  Synchronous. */
pf_status pf_analyze(pf_ctx *ctx, pf_symbolic_info *info);

/* Copies the symbolic result of matrix `which` to caller arrays sized from
 * pf_symbolic_info: perm[n] (elimination step -> local index), parent[n]
 * (step -> parent step, -1 = root), level[n] (1 = leaf), Lp[n+1], Li[nnz_l]
 * (strict lower pattern of L by column, rows ascending, in step numbering).
 * Any pointer may be NULL.  Synchronous. */
pf_status pf_get_symbolic(const pf_ctx *ctx, int32_t which, int32_t *perm, int32_t *parent,
                          int32_t *level, int64_t *Lp, int32_t *Li);

/* Elimination tree and level sets of a filled pattern on the GPU (Section
 * II.B: FormEliminationTree and the leaf-peeling partition of Table I), for
 * workloads whose topology changes: from the strict-lower pattern of L by
 * column, Lp_dev[n + 1] (int64) and Li_dev[Lp[n]] (int32 rows; caller-owned
 * device arrays, e.g. pf_get_symbolic's uploaded), it writes parent_dev[j] =
 * the smallest row i > j of column j (-1 for a root), level_dev[j] = 1 for a
 * leaf, else 1 + the largest level of j's children, and nlev_dev[0] = the
 * number of levels -- the same numbers as pf_get_symbolic's.  scratch_dev:
 * 3 n int32 of caller-owned device memory.  PF_ERR_ARG for n < 1 or a NULL
 * pointer, PF_ERR_CUDA for a failed launch.  Asynchronous on `stream`. */
pf_status pf_etree_levels_device(int32_t n, const int64_t *Lp_dev, const int32_t *Li_dev,
                                 int32_t *parent_dev, int32_t *level_dev, int32_t *nlev_dev,
                                 int32_t *scratch_dev, void *stream);

/* Defines a batch of ncase >= 1 cases sharing the topology.  load_scale
 * [ncase][nbus] (host, NULL = all 1) multiplies pd and qd of every PQ bus of
 * a case; outage[ncase] (host, NULL = none) names a branch taken out of
 * service in that case (-1 = none).  Outages keep the symbolic pattern.
 * Replaces any previous batch.  A call with the same cases as the current
 * batch (count and outages) keeps its device arrays, factors and CUDA graph
 * and only forms the specified injections again.  PF_ERR_ARG for an outage
 * out of range or a non-finite load scale (then the batch's injections are
 * unchanged).  Synchronous. */
pf_status pf_set_cases(pf_ctx *ctx, int32_t ncase, const double *load_scale,
                       const int32_t *outage);

/* Overrides the specified injections of the current batch with device
 * arrays psp_dev / qsp_dev [ncase][nbus] (Psp used at non-slack buses, Qsp at
 * PQ buses; other entries ignored), e.g. to differentiate the power flow with
 * respect to them.  Asynchronous. */
pf_status pf_set_injections(pf_ctx *ctx, const double *psp_dev, const double *qsp_dev,
                            void *stream);

/* Assembles the bus admittance matrix (Section III.A) and the values of B'
 * or B'' for every case and factorises them level by level (Section III.B):
 * A = L D L^T with unit L.  precision selects FP64 or FP32 factor storage.
 * Asynchronous; a singular or non-finite pivot is recorded in the per-case
 * status read by pf_get_factor / pf_case_status. */
pf_status pf_factor(pf_ctx *ctx, int32_t which, int32_t precision, void *stream);

/* Copies case c's factor of matrix `which` to the host: D[n] and Lx[nnz_l]
 * in step numbering, as doubles whatever the storage precision, and its
 * factor status (PF_OK, PF_ERR_SINGULAR or PF_ERR_NONFINITE).  Synchronous. */
pf_status pf_get_factor(pf_ctx *ctx, int32_t which, int32_t precision, int32_t c, double *D,
                        double *Lx, int32_t *status);

/* Solves A x = rhs in place for the first ncase cases with the factor of the
 * given precision (forward substitution, normalisation y = z / d (Eq. 4),
 * back substitution, Section III.C).  rhs_inout_dev is [ncase][n] double in
 * local order.  transpose is accepted for symmetry (B' and B'' are
 * symmetric).  Asynchronous. */
pf_status pf_solve(pf_ctx *ctx, int32_t which, int32_t precision, int32_t transpose,
                   double *rhs_inout_dev, int32_t ncase, void *stream);

/* Nodal P/Q mismatch (Section II.A) of the first ncase cases at the states
 * vm_dev/va_dev [ncase][nbus]: dp_dev/dq_dev [ncase][nbus] receive
 * Psp - P (non-slack, else 0) and Qsp - Q (PQ, else 0); maxmis_dev[ncase]
 * receives max |.|.  Uses each case's outage and load scale.  Asynchronous. */
pf_status pf_mismatch(pf_ctx *ctx, const double *vm_dev, const double *va_dev, double *dp_dev,
                      double *dq_dev, double *maxmis_dev, int32_t ncase, void *stream);

/* Runs the power flow of every case of the batch to opts->tol on the device
 * and returns per-case results in res_host[ncase].  vm_dev/va_dev
 * [ncase][nbus] hold the start (unless flat_start) and receive the final
 * state.  Assembly, factor, substitutions, mismatch and convergence checks
 * all run in device kernels; the call returns after the device is done.
 * Returns PF_OK when every case converged, else the first failing status. */
pf_status pf_run_to_tol(pf_ctx *ctx, const pf_run_opts *opts, double *vm_dev, double *va_dev,
                        pf_case_result *res_host, void *stream);

/* Kernel kinds counted by the profiling hooks. */
enum {
    PF_K_YBUS = 0,     /* admittance matrix and XB B' assembly (Section III.A) */
    PF_K_SPEC = 1,     /* specified injections of every case */
    PF_K_ASSEMBLE = 2, /* B' / B'' values of every factor instance */
    PF_K_FACTOR = 3,   /* level-scheduled LDL^T (Section III.B) */
    PF_K_SOLVE = 4,    /* level-scheduled substitutions (Section III.C) */
    PF_K_MISMATCH = 5, /* nodal injections and mismatch (Section II.A) */
    PF_K_RUN = 6,      /* the power-flow iteration kernel of pf_run_to_tol */
    PF_K_COUNT = 7
};

/* Turns per-launch CUDA-event timing of this context's kernels on (1) or off
 * (0).  Launch counts are always kept.  Synchronous. */
pf_status pf_set_profiling(pf_ctx *ctx, int32_t on);

/* CUDA graphs of repeated runs (on by default): a fast decoupled
 * pf_run_to_tol on the block or cluster engine whose arguments (state
 * pointers, options, tuning, batch) repeat those of the previous call is
 * captured once into a CUDA graph of its device work -- admittance and
 * matrix assembly, both factorisations, the low-rank or tail-inverse
 * preparation, the iteration kernel -- and later identical calls launch that
 * graph instead of the individual kernels.  Off (0): every call launches its
 * kernels directly.  Runs with profiling on are always direct.  Not part of
 * the paper's method: it only removes launch overhead.  Synchronous. */
pf_status pf_set_graphs(pf_ctx *ctx, int32_t on);

/* Launch count and summed device time (ms, 0 unless profiling was on) of one
 * kernel kind since the last reset; reset = 1 clears both afterwards.
 * Synchronises with the recorded events. */
pf_status pf_get_profile(pf_ctx *ctx, int32_t kind, int64_t *launches, double *total_ms,
                         int32_t reset);

/* Adjoint of the Newton-Raphson power flow (transposed solve with the
 * factors of the last PF_NR pf_run_to_tol of the same precision, refined in
 * FP64 against the exact Jacobian at the given state).  For every case c,
 * with J the Jacobian of the mismatch F(x) = Psp - P(x) at the state
 * vm_dev/va_dev [ncase][nbus]: solves J^T y = g, where g holds dObj/dtheta
 * (gva_dev) of every non-slack bus and dObj/dV (gvm_dev) of every PQ bus
 * (other entries are ignored), and writes dObj/dPsp = y_P to dJdP_dev and
 * dObj/dQsp = y_Q to dJdQ_dev [ncase][nbus] (0 at the slack, dJdQ 0 at PV
 * buses).  If no Newton factors exist yet the Jacobian at the state is
 * factorised first.  Returns after the device is done; per-case status in
 * res_host[ncase]. */
pf_status pf_adjoint(pf_ctx *ctx, int32_t precision, const double *vm_dev, const double *va_dev,
                     const double *gva_dev, const double *gvm_dev, double *dJdP_dev,
                     double *dJdQ_dev, pf_case_result *res_host, void *stream);

/* Objective J = sum_i (V_i - 1)^2 + sum_i P_i (the total active losses) of
 * every case at vm_dev/va_dev [ncase][nbus] into J_dev[ncase], and its
 * gradient: gva_dev[ncase][nbus] = dJ/dtheta_k, gvm_dev[ncase][nbus] =
 * dJ/dV_k for every bus.  Asynchronous. */
pf_status pf_objective(pf_ctx *ctx, const double *vm_dev, const double *va_dev, double *J_dev,
                       double *gva_dev, double *gvm_dev, void *stream);

/* Branch flows and losses after a solve (the per-branch split of the nodal
 * injections of Section II.A; the losses are the second term of the adjoint
 * objective).  For case c and branch k (pf_create's order),
 * flows_dev[(c * nbranch + k) * 4 + {0, 1, 2, 3}] = (P_f, Q_f, P_t, Q_t): the
 * complex power entering the branch at its from and at its to end, with the
 * pi model of the admittance matrix (tap on the from side).  The case's
 * outaged branch and out-of-service branches carry zero.  loss_dev[c] = the
 * sum over branches of P_f + P_t plus the shunt consumption sum gs V^2 (the
 * total active loss).  vm_dev / va_dev: [ncase][nbus] device states (as
 * written by pf_run_to_tol).  PF_ERR_ARG for a NULL pointer or ncase outside
 * 1 .. the cases set.  Asynchronous on `stream`. */
pf_status pf_branch_flows(pf_ctx *ctx, const double *vm_dev, const double *va_dev, int32_t ncase,
                          double *flows_dev, double *loss_dev, void *stream);

/* Project autotuner: runs pf_run_to_tol with opts (engine AUTO) under every
 * applicable mapping of pf_tuning -- engines for FDPF batches, cluster sizes
 * for single cases, block sizes for one block per case, the two factor
 * forms, the two tail forms, the two outage forms -- `reps` times
 * each after one untimed run, times them with CUDA events on `stream`, and
 * keeps the fastest mapping whose cases all converged; it becomes the
 * context's tuning (used by later runs) and is written to *out.  vm_dev,
 * va_dev as for pf_run_to_tol (overwritten).  PF_ERR_ARG for reps < 1 or bad
 * options; the status of pf_run_to_tol when no mapping converges.
 * Synchronous. */
pf_status pf_autotune(pf_ctx *ctx, const pf_run_opts *opts, double *vm_dev, double *va_dev,
                      int32_t reps, pf_tuning *out, void *stream);

/* Reads or replaces the context's tuning.  PF_ERR_ARG for a field out of
 * range.  Synchronous, host only. */
pf_status pf_get_tuning(const pf_ctx *ctx, pf_tuning *out);
pf_status pf_set_tuning(pf_ctx *ctx, const pf_tuning *tuning);

/* Message of the last failing call on this context (never NULL). */
const char *pf_last_error(const pf_ctx *ctx);

/* Copies the base-case admittance matrix: rowptr[nbus+1], col[nnz], G[nnz],
 * B[nnz] (CSR, columns ascending, diagonal present).  Synchronous. */
pf_status pf_get_ybus(pf_ctx *ctx, int32_t *rowptr, int32_t *col, double *G, double *B);

/* Largest nbus accepted by pf_mismatch_static. */
#define PF_STATIC_MAX_BUS 131072

/* Allocation-free P/Q mismatch of one case (the paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory,
 * e.g. processes that reserve their whole device budget at start-up and
 * forbid later allocation, or applications whose own allocator owns the GPU).
 * It needs no context: every input and output is caller-owned device memory
 * -- the admittance matrix rowptr[nbus+1], col[nnz], G[nnz], B[nnz] (CSR as
 * returned by pf_get_ybus), btype[nbus] (PF_BUS_*), specified injections
 * psp[nbus] = pg - pd and qsp[nbus] = -qd, the state vm/va[nbus]; outputs
 * dp/dq[nbus] and maxmis[1] exactly as pf_mismatch computes them for one case
 * without outage.  It calls no cudaMalloc, cudaFree or allocating routine:
 * its only intermediate, the rectangular voltages, lives in a fixed device
 * array of 2 * PF_STATIC_MAX_BUS doubles (2 MiB) that every GPU which loads
 * the library holds until the process exits.  The first call on a device
 * looks up that array's device address with the device current, so make
 * that first call before any stream capture.  All calls share the array and
 * it keeps the last call's contents: calls whose kernels can overlap on the
 * GPU (other streams, other host threads) race and must be serialised by
 * the caller.  maxmis is cleared by the call.  Returns PF_ERR_ARG when nbus is
 * < 1 or > PF_STATIC_MAX_BUS or a pointer is NULL, PF_ERR_CUDA when the
 * address look-up or a launch fails.  Asynchronous on `stream`. */
pf_status pf_mismatch_static(int32_t nbus, const int32_t *rowptr_dev, const int32_t *col_dev,
                             const double *G_dev, const double *B_dev, const int32_t *btype_dev,
                             const double *psp_dev, const double *qsp_dev, const double *vm_dev,
                             const double *va_dev, double *dp_dev, double *dq_dev,
                             double *maxmis_dev, void *stream);

/* Releases the context and all its device memory.  NULL is accepted. */
void pf_destroy(pf_ctx *ctx);

/* ---------------------------------------------------------------- packs
 * An uneven multi-grid batch: many independent grids of different sizes,
 * each with its own ordering, elimination tree and level sets (its own
 * context), solved by one persistent launch in which the thread blocks take
 * the grids largest first (the batched serving pattern of the problem
 * statement applied across grids; the paper solves one grid per call,
 * Section III).  The pack does not own the contexts. */
typedef struct pf_pack pf_pack;

/* Creates a pack over grids[0..ngrid).  Every context must have been
 * analysed; the pack keeps the pointers, so the contexts must outlive it.
 * PF_ERR_ARG for ngrid < 1, a NULL or repeated context, or a factor column
 * of more than 255 strict-lower entries (pf_symbolic_info.max_col);
 * PF_ERR_STATE for a context not analysed.  Synchronous. */
pf_status pf_pack_create(pf_ctx *const *grids, int32_t ngrid, pf_pack **out);

/* Runs every grid of the pack to opts->tol with the fast decoupled method
 * (opts->method must be PF_FDPF; precision, tolerance, iteration and
 * refinement options as for pf_run_to_tol; engine is ignored).  For each
 * grid it assembles the admittance matrix and B', B'' of its one case
 * (pf_set_cases with ncase 1, or never called); one dependency-driven launch
 * factorises every grid's B' and B'' (Section III.B), then one launch
 * iterates all grids.  vm_dev / va_dev are caller-owned device arrays of
 * sum(nbus) doubles, the grids' buses concatenated in pack order, with the
 * start state read when opts->flat_start is 0 and the solution written;
 * res_host[ngrid] receives each grid's outcome.  Returns PF_OK when every
 * grid converged, else the first failing grid's status (all results are
 * still written).  Synchronous with respect to the host; work is issued on
 * `stream`. */
pf_status pf_pack_run(pf_pack *pack, const pf_run_opts *opts, double *vm_dev, double *va_dev,
                      pf_case_result *res_host, void *stream);

/* Message of the last failing pack call (never NULL). */
const char *pf_pack_last_error(const pf_pack *pack);

/* Releases the pack's own device memory (not the contexts).  NULL is accepted. */
void pf_pack_destroy(pf_pack *pack);

#ifdef __cplusplus
}
#endif

#endif /* GBPF_H */
