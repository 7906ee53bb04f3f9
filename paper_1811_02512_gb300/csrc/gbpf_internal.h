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

// Symbolic data of one factorised matrix (B' or B''), device copies.
// Numbering: "step" k = position in the elimination order; every array below
// is in step numbering unless named otherwise.
struct DevMat {
    int n = 0;           // dimension (buses in the matrix)
    int nnz_l = 0;       // strict-lower nonzeros of L
    int nlev = 0;        // levels of the elimination tree
    int max_col = 0;     // largest column count of L
    int64_t nupd = 0;    // entries of the update map
    int stride = 0;      // per-instance value stride: n diagonal slots + nnz_l, padded
    int *bus = nullptr;      // [n]     step -> global bus
    int *perm = nullptr;     // [n]     step -> local index (ascending-bus order)
    int *Lp = nullptr;       // [n+1]   column pointers of L
    int *Li = nullptr;       // [nnz_l] row (step) of every L entry, ascending per column
    int *Rp = nullptr;       // [n+1]   row pointers of L (row lists)
    int *Rk = nullptr;       // [nnz_l] column (step) of every row-list entry, ascending
    int *Rpos = nullptr;     // [nnz_l] position in the column-ordered L values
    int *lvl_ptr = nullptr;  // [nlev+1]
    int *lvl_cols = nullptr; // [n]     steps grouped by level (ascending), ascending within
    int *uoff = nullptr;     // [nnz_l+1] start of each row-list entry's map in umap
    int *umap = nullptr;     // [nupd]  column-relative target (0 = diagonal, 1 + t = t-th L entry)
    int *src = nullptr;      // [n + nnz_l] Ybus-pattern position feeding each slot, -1 = fill
    int *step_of_bus = nullptr; // [nbus] global bus -> step, -1 if not in the matrix
    int *br_slot = nullptr;  // [nbranch*3] slots of (diag f, diag t, L(f,t)) or -1
};

// Host copy of the symbolic data of one matrix.
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
    std::vector<int> lvl_ptr, lvl_cols;
    std::vector<int> Rp, Rk, Rpos;
    std::vector<int> uoff, umap;
    std::vector<int> src;
    std::vector<int> step_of_bus;
    std::vector<int> br_slot;
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
};

struct DevCases {
    int ncase = 0;
    int ninst = 1;            // factor instances: 0 = base, 1.. = outage cases
    int *outage = nullptr;    // [ncase] branch or -1
    int *inst = nullptr;      // [ncase] factor instance of each case
    int *inst_outage = nullptr; // [ninst] branch of each instance (-1 for base)
    double *Psp = nullptr, *Qsp = nullptr; // [ncase][nbus]
};

struct Workspace {
    // factor storage per matrix and precision: [ninst][stride]
    double *A[2] = {nullptr, nullptr};       // assembled values (FP64), per instance
    double *F64[2] = {nullptr, nullptr};
    float *F32[2] = {nullptr, nullptr};
    int *fstatus[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}}; // [mat][prec] per instance
    bool factored[2][2] = {{false, false}, {false, false}};
    int ninst_alloc = 0;
    // per-case scratch
    double *ef = nullptr;     // [ncase][2*nbus] rectangular voltages
    double *vec = nullptr;    // [ncase][2*nbus] global solve vectors when they exceed shared memory
    int *cstatus = nullptr;   // [ncase] run status
    pf_case_result *res = nullptr; // [ncase]
    int ncase_alloc = 0;
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
    std::vector<int> ydiag, inc_ptr, inc_br, inc_side, inc_pos, br_pos;
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    std::string err;
    std::vector<void *> allocations;  // everything owned by the context
};

namespace gbpf {

// Launch wrappers implemented in gbpf_kernels.cu.  All return cudaError_t of
// the launch (asynchronous errors surface at the next synchronising call).
cudaError_t launch_ybus(const DevNet &dn, cudaStream_t s);
cudaError_t launch_case_spec(const DevNet &dn, const DevCases &dc, const double *load_scale_dev,
                             cudaStream_t s);
cudaError_t launch_assemble_slots(const DevNet &dn, const DevCases &dc, const DevMat &m, int which,
                                  double *A, cudaStream_t s);
cudaError_t launch_factor(const DevMat &m, int prec, const double *A, void *F, int ninst,
                          int *fstatus, cudaStream_t s);
cudaError_t launch_solve(const DevMat &m, int prec, const void *F, const int *inst_of_case,
                         double *rhs, int ncase, void *gvec, size_t smem_optin, cudaStream_t s);
cudaError_t launch_mismatch(const DevNet &dn, const DevCases &dc, const double *vm, const double *va,
                            double *dp, double *dq, double *maxmis, double *ef, int ncase,
                            cudaStream_t s);
cudaError_t launch_fdpf(const DevNet &dn, const DevCases &dc, const DevMat *m, int prec,
                        const void *F0, const void *F1, const int *fstat0, const int *fstat1,
                        const pf_run_opts &o, double *vm, double *va, double *ef, double *vec,
                        pf_case_result *res, size_t smem_optin, cudaStream_t s);

}  // namespace gbpf
