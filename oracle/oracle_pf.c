/*
 * oracle_pf.c -- plain FP64 CPU oracle for the graph-based power flow of
 * "Graph Based Power Flow Calculation for Energy Management System"
 * (arxiv 1811.02512).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, obviously correct reference
 * that the CUDA library is checked against.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it; the library never
 * does, and the two share no code, header or table.
 *
 * Everything is sequential double precision.  Each routine cites the passage
 * of the paper it restates:
 *   Section III.A  FormMatrixA            -> or_ybus_pattern / or_ybus_values
 *   Section II.A   nodal injections       -> or_injections / or_mismatch
 *   Section II.B.1 FormFilledGraph        -> or_filled_graph
 *   Section II.B.2 FormEliminationTree    -> or_etree
 *   Section II.B   FormHierarchicalPartition, Table I -> or_levels
 *   Section III.B  FactorizeGraphA, Eqs. 1-3 -> or_lu
 *   Section III.C  forward / normalisation (Eq. 4) / backward -> or_lu_solve
 *   Section III    Newton-Raphson and fast decoupled iterations -> or_power_flow
 * The ordering (exact minimum degree), the etree-merge symbolic
 * factorisation and the adjoint are not in the paper; they are written from
 * their textbook definitions.
 *
 * Readings of the paper (where it is garbled or silent) that this file takes:
 *  - "a_ii += a_ij" in FormMatrixA is the pi-model diagonal accumulation:
 *    Y_ff += (y + jb/2)/t^2, Y_tt += y + jb/2, Y_ft = Y_tf -= y/t,
 *    Y_ii += gs + j bs (tap t on the from side, no phase shift).
 *  - "z_i = b_i - l_ij z_i" means z_i = b_i - sum_{j<i} l_ij z_j and
 *    "x_i = y_i - u_ij x_i" means x_i = y_i - sum_{j>i} u_ij x_j.
 *  - the numeric factor is LU without pivoting on the filled pattern; for a
 *    symmetric matrix D = diag(U) and U = D L^T (Eq. 1-3).
 *  - fast decoupled uses the XB scheme: B'_ij = -1/x_ij, B'_ii = sum 1/x_ij
 *    on non-slack buses; B'' = -Im(Ybus) on PQ buses.
 *  - Newton-Raphson is polar with unknowns (theta_i, V_i) per non-slack bus;
 *    the V unknown of a PV bus is pinned by an identity row and column.
 *  - convergence: max(|dP| over non-slack, |dQ| over PQ) <= tol, checked
 *    before every (half-)step.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_ISLAND 2
#define OR_ERR_SINGULAR 3
#define OR_ERR_NONFINITE 4
#define OR_ERR_NOT_CONVERGED 5
#define OR_ERR_OOM 8

#define OR_PQ 1
#define OR_PV 2
#define OR_SLACK 3

#define OR_FDPF 1
#define OR_NR 2

/* ------------------------------------------------------------------ sets */

/* A growable sorted set of ints (adjacency list of one vertex). */
typedef struct {
    int *a;
    int n, cap;
} iset;

static int iset_find(const iset *s, int v) {
    int lo = 0, hi = s->n;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (s->a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int iset_has(const iset *s, int v) {
    int p = iset_find(s, v);
    return p < s->n && s->a[p] == v;
}

/* returns 1 if inserted, 0 if present, -1 on allocation failure */
static int iset_insert(iset *s, int v) {
    int p = iset_find(s, v);
    if (p < s->n && s->a[p] == v) return 0;
    if (s->n == s->cap) {
        int nc = s->cap ? 2 * s->cap : 4;
        int *na = (int *)realloc(s->a, sizeof(int) * (size_t)nc);
        if (!na) return -1;
        s->a = na;
        s->cap = nc;
    }
    memmove(s->a + p + 1, s->a + p, sizeof(int) * (size_t)(s->n - p));
    s->a[p] = v;
    s->n++;
    return 1;
}

static void iset_remove(iset *s, int v) {
    int p = iset_find(s, v);
    if (p < s->n && s->a[p] == v) {
        memmove(s->a + p, s->a + p + 1, sizeof(int) * (size_t)(s->n - p - 1));
        s->n--;
    }
}

static void isets_free(iset *s, int n) {
    if (!s) return;
    for (int i = 0; i < n; i++) free(s[i].a);
    free(s);
}

/* Build adjacency sets of an undirected graph given in CSR (self loops dropped). */
static iset *isets_from_csr(int n, const int *adjp, const int *adji) {
    iset *s = (iset *)calloc((size_t)(n > 0 ? n : 1), sizeof(iset));
    if (!s) return NULL;
    for (int i = 0; i < n; i++)
        for (int p = adjp[i]; p < adjp[i + 1]; p++) {
            int j = adji[p];
            if (j == i) continue;
            if (iset_insert(&s[i], j) < 0 || iset_insert(&s[j], i) < 0) {
                isets_free(s, n);
                return NULL;
            }
        }
    return s;
}

/* --------------------------------------------------- Section III.A: Ybus */

/* Pattern of the bus admittance matrix: for every bus its own diagonal and
 * one entry per adjacent bus (every branch, in service or not, keeps its
 * slot).  CSR with ascending columns.  rowptr[n+1], col[<= n + 2m].
 * Returns nnz or -1. */
int or_ybus_pattern(int n, int m, const int *f, const int *t, int *rowptr, int *col) {
    iset *s = (iset *)calloc((size_t)(n > 0 ? n : 1), sizeof(iset));
    if (!s) return -1;
    for (int i = 0; i < n; i++)
        if (iset_insert(&s[i], i) < 0) { isets_free(s, n); return -1; }
    for (int k = 0; k < m; k++) {
        if (f[k] < 0 || f[k] >= n || t[k] < 0 || t[k] >= n || f[k] == t[k]) {
            isets_free(s, n);
            return -1;
        }
        if (iset_insert(&s[f[k]], t[k]) < 0 || iset_insert(&s[t[k]], f[k]) < 0) {
            isets_free(s, n);
            return -1;
        }
    }
    int nnz = 0;
    rowptr[0] = 0;
    for (int i = 0; i < n; i++) {
        for (int q = 0; q < s[i].n; q++) col[nnz++] = s[i].a[q];
        rowptr[i + 1] = nnz;
    }
    isets_free(s, n);
    return nnz;
}

static int csr_pos(const int *rowptr, const int *col, int i, int j) {
    int lo = rowptr[i], hi = rowptr[i + 1];
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (col[mid] < j) lo = mid + 1; else hi = mid;
    }
    return (lo < rowptr[i + 1] && col[lo] == j) ? lo : -1;
}

/* FormMatrixA (Section III.A): accumulate the pi-model of every in-service
 * branch and the bus shunts into Y = G + jB on the given pattern. */
int or_ybus_values(int n, int m, const int *f, const int *t, const double *r, const double *x,
                   const double *b, const double *tap, const int *status, const double *gs,
                   const double *bs, const int *rowptr, const int *col, double *G, double *B) {
    int nnz = rowptr[n];
    for (int p = 0; p < nnz; p++) { G[p] = 0.0; B[p] = 0.0; }
    for (int k = 0; k < m; k++) {
        if (!status[k]) continue;
        double den = r[k] * r[k] + x[k] * x[k];
        if (!(den > 0.0)) return OR_ERR_ARG;
        double ys_re = r[k] / den, ys_im = -x[k] / den; /* y = 1/(r + jx) */
        double tt = (tap[k] == 0.0) ? 1.0 : tap[k];
        int ff = csr_pos(rowptr, col, f[k], f[k]);
        int tt_ = csr_pos(rowptr, col, t[k], t[k]);
        int ft = csr_pos(rowptr, col, f[k], t[k]);
        int tf = csr_pos(rowptr, col, t[k], f[k]);
        if (ff < 0 || tt_ < 0 || ft < 0 || tf < 0) return OR_ERR_ARG;
        G[ff] += ys_re / (tt * tt);
        B[ff] += (ys_im + 0.5 * b[k]) / (tt * tt);
        G[tt_] += ys_re;
        B[tt_] += ys_im + 0.5 * b[k];
        G[ft] -= ys_re / tt;
        B[ft] -= ys_im / tt;
        G[tf] -= ys_re / tt;
        B[tf] -= ys_im / tt;
    }
    for (int i = 0; i < n; i++) {
        int d = csr_pos(rowptr, col, i, i);
        G[d] += gs[i];
        B[d] += bs[i];
    }
    return OR_OK;
}

/* XB fast-decoupled B' on the Ybus pattern: B'_ij = -1/x_ij (summed over
 * parallel in-service branches), B'_ii = sum_j 1/x_ij.  Resistance, charging,
 * taps and shunts are ignored (Section III, fast decoupled power flow). */
int or_bprime_values(int n, int m, const int *f, const int *t, const double *x, const int *status,
                     const int *rowptr, const int *col, double *Bp) {
    for (int p = 0; p < rowptr[n]; p++) Bp[p] = 0.0;
    for (int k = 0; k < m; k++) {
        if (!status[k]) continue;
        if (x[k] == 0.0) return OR_ERR_ARG;
        double bb = 1.0 / x[k];
        Bp[csr_pos(rowptr, col, f[k], f[k])] += bb;
        Bp[csr_pos(rowptr, col, t[k], t[k])] += bb;
        Bp[csr_pos(rowptr, col, f[k], t[k])] -= bb;
        Bp[csr_pos(rowptr, col, t[k], f[k])] -= bb;
    }
    return OR_OK;
}

/* ------------------------------------ Section II.A: nodal injections */

/* S_i = V_i conj(sum_k Y_ik V_k) for every bus, with V = vm e^{j va}. */
void or_injections(int n, const int *rowptr, const int *col, const double *G, const double *B,
                   const double *vm, const double *va, double *P, double *Q) {
    for (int i = 0; i < n; i++) {
        double ire = 0.0, iim = 0.0;
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            int k = col[p];
            double ek = vm[k] * cos(va[k]), fk = vm[k] * sin(va[k]);
            ire += G[p] * ek - B[p] * fk;
            iim += G[p] * fk + B[p] * ek;
        }
        double ei = vm[i] * cos(va[i]), fi = vm[i] * sin(va[i]);
        P[i] = ei * ire + fi * iim;
        Q[i] = fi * ire - ei * iim;
    }
}

/* Mismatch and convergence check (Section II.A): dP = Psp - P at non-slack
 * buses, dQ = Qsp - Q at PQ buses, zero elsewhere; returns max |.|. */
double or_mismatch(int n, const int *btype, const double *Psp, const double *Qsp,
                   const double *P, const double *Q, double *dP, double *dQ) {
    double mx = 0.0;
    for (int i = 0; i < n; i++) {
        dP[i] = (btype[i] != OR_SLACK) ? Psp[i] - P[i] : 0.0;
        dQ[i] = (btype[i] == OR_PQ) ? Qsp[i] - Q[i] : 0.0;
        double a = fabs(dP[i]), c = fabs(dQ[i]);
        if (!(a <= mx)) mx = a;       /* NaN propagates into mx */
        if (!(c <= mx)) mx = c;
    }
    return mx;
}

/* -------------------------------------- ordering: exact minimum degree */

typedef struct { int deg, v; } hent;

static int hless(hent a, hent b) { return a.deg < b.deg || (a.deg == b.deg && a.v < b.v); }

typedef struct { hent *h; int n, cap; } heap;

static int heap_push(heap *H, hent e) {
    if (H->n == H->cap) {
        int nc = H->cap ? 2 * H->cap : 64;
        hent *nh = (hent *)realloc(H->h, sizeof(hent) * (size_t)nc);
        if (!nh) return -1;
        H->h = nh;
        H->cap = nc;
    }
    int i = H->n++;
    H->h[i] = e;
    while (i > 0) {
        int p = (i - 1) / 2;
        if (!hless(H->h[i], H->h[p])) break;
        hent tmp = H->h[i]; H->h[i] = H->h[p]; H->h[p] = tmp;
        i = p;
    }
    return 0;
}

static hent heap_pop(heap *H) {
    hent top = H->h[0];
    H->h[0] = H->h[--H->n];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, s = i;
        if (l < H->n && hless(H->h[l], H->h[s])) s = l;
        if (r < H->n && hless(H->h[r], H->h[s])) s = r;
        if (s == i) break;
        hent tmp = H->h[i]; H->h[i] = H->h[s]; H->h[s] = tmp;
        i = s;
    }
    return top;
}

/* Exact minimum degree on the elimination graph: at every step eliminate the
 * remaining vertex with the fewest remaining neighbours (fill included), ties
 * to the smallest index; its neighbours become a clique.  perm[k] is the
 * vertex eliminated at step k.  Returns 0 or an error code. */
int or_min_degree(int n, const int *adjp, const int *adji, int *perm) {
    iset *adj = isets_from_csr(n, adjp, adji);
    if (!adj && n > 0) return OR_ERR_OOM;
    char *gone = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    heap H = {0, 0, 0};
    int rc = OR_OK;
    for (int v = 0; v < n; v++)
        if (heap_push(&H, (hent){adj[v].n, v})) { rc = OR_ERR_OOM; goto done; }
    for (int step = 0; step < n; step++) {
        hent e;
        do {
            e = heap_pop(&H);
        } while (gone[e.v] || e.deg != adj[e.v].n);
        int v = e.v;
        perm[step] = v;
        gone[v] = 1;
        iset nb = adj[v];
        for (int a = 0; a < nb.n; a++) {
            int u = nb.a[a];
            iset_remove(&adj[u], v);
            for (int c = 0; c < nb.n; c++)
                if (c != a && iset_insert(&adj[u], nb.a[c]) < 0) { rc = OR_ERR_OOM; goto done; }
        }
        for (int a = 0; a < nb.n; a++)
            if (heap_push(&H, (hent){adj[nb.a[a]].n, nb.a[a]})) { rc = OR_ERR_OOM; goto done; }
        free(adj[v].a);
        adj[v].a = NULL;
        adj[v].n = adj[v].cap = 0;
    }
done:
    free(H.h);
    free(gone);
    isets_free(adj, n);
    return rc;
}

/* ----------------------------------------- Section II.B.1: fill-ins */

/* FormFilledGraph taken literally: nodes in order i = 0..n-1; every pair of
 * neighbours j, k of i with j > i and k > i becomes adjacent (a fill-in when
 * it was not).  Fill created at step i is adjacency at later steps, so the
 * outer loop is sequential.  Output: strict lower pattern of L by column
 * (column i = neighbours of i greater than i, ascending).  Returns nnz(L),
 * -1 on allocation failure, -2 if cap is too small. */
long long or_filled_graph(int n, const int *adjp, const int *adji, long long *Lp, int *Li,
                          long long cap) {
    iset *adj = isets_from_csr(n, adjp, adji);
    if (!adj && n > 0) return -1;
    for (int i = 0; i < n; i++) {
        int s = iset_find(&adj[i], i + 1); /* neighbours > i */
        for (int a = s; a < adj[i].n; a++)
            for (int c = a + 1; c < adj[i].n; c++) {
                int j = adj[i].a[a], k = adj[i].a[c];
                if (iset_insert(&adj[j], k) < 0 || iset_insert(&adj[k], j) < 0) {
                    isets_free(adj, n);
                    return -1;
                }
            }
    }
    long long nz = 0;
    Lp[0] = 0;
    for (int i = 0; i < n; i++) {
        for (int a = iset_find(&adj[i], i + 1); a < adj[i].n; a++) {
            if (nz >= cap) { isets_free(adj, n); return -2; }
            Li[nz++] = adj[i].a[a];
        }
        Lp[i + 1] = nz;
    }
    isets_free(adj, n);
    return nz;
}

/* Second, independent symbolic factorisation: the elimination tree from the
 * matrix pattern (Liu's ancestor walk) and then every column structure as
 * struct(A_j, rows > j) united with struct(L_c) minus {j} over the children
 * c of j.  Same output format as or_filled_graph. */
long long or_symbolic_etree(int n, const int *adjp, const int *adji, long long *Lp, int *Li,
                            long long cap) {
    int *parent = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *anc = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *mark = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *head = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *next = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    long long ret = -1;
    iset *colset = NULL;
    if (!parent || !anc || !mark || !head || !next) goto out;
    for (int i = 0; i < n; i++) { parent[i] = -1; anc[i] = -1; mark[i] = -1; head[i] = -1; }
    for (int i = 0; i < n; i++)
        for (int p = adjp[i]; p < adjp[i + 1]; p++) {
            int k = adji[p];
            if (k >= i) continue;
            while (k != -1 && k != i) {
                int nx = anc[k];
                anc[k] = i;
                if (nx == -1) parent[k] = i;
                k = nx;
            }
        }
    /* children lists, ascending */
    for (int j = n - 1; j >= 0; j--)
        if (parent[j] >= 0) { next[j] = head[parent[j]]; head[parent[j]] = j; }
    colset = (iset *)calloc((size_t)(n > 0 ? n : 1), sizeof(iset));
    if (!colset) goto out;
    for (int j = 0; j < n; j++) {
        for (int p = adjp[j]; p < adjp[j + 1]; p++)
            if (adji[p] > j && iset_insert(&colset[j], adji[p]) < 0) goto out;
        for (int c = head[j]; c != -1; c = next[c])
            for (int q = 0; q < colset[c].n; q++)
                if (colset[c].a[q] != j && iset_insert(&colset[j], colset[c].a[q]) < 0) goto out;
    }
    {
        long long nz = 0;
        Lp[0] = 0;
        for (int j = 0; j < n; j++) {
            for (int q = 0; q < colset[j].n; q++) {
                if (nz >= cap) { ret = -2; goto out; }
                Li[nz++] = colset[j].a[q];
            }
            Lp[j + 1] = nz;
        }
        ret = nz;
    }
out:
    isets_free(colset, n);
    free(parent); free(anc); free(mark); free(head); free(next);
    return ret;
}

/* ------------------------------------ Section II.B.2: elimination tree */

/* FormEliminationTree: parent of i is the smallest neighbour j > i in the
 * filled graph, i.e. the first row of column i of L; -1 for a root. */
void or_etree(int n, const long long *Lp, const int *Li, int *parent) {
    for (int i = 0; i < n; i++) {
        int best = -1;
        for (long long p = Lp[i]; p < Lp[i + 1]; p++)
            if (Li[p] > i && (best < 0 || Li[p] < best)) best = Li[p];
        parent[i] = best;
    }
}

/* -------------------- Section II.B: FormHierarchicalPartition (Table I) */

/* Repeated leaf peeling: all current leaves get the current level (leaves of
 * the original tree are level 1) and are removed together; the level then
 * advances.  Returns the number of levels. */
int or_levels(int n, const int *parent, int *level) {
    int *kids = (int *)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
    char *removed = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int *batch = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!kids || !removed || !batch) { free(kids); free(removed); free(batch); return -1; }
    for (int i = 0; i < n; i++)
        if (parent[i] >= 0) kids[parent[i]]++;
    int remaining = n, lev = 0;
    while (remaining > 0) {
        lev++;
        int nb = 0;
        for (int i = 0; i < n; i++)
            if (!removed[i] && kids[i] == 0) batch[nb++] = i;
        if (nb == 0) { lev = -1; break; } /* not a forest */
        for (int q = 0; q < nb; q++) {
            level[batch[q]] = lev;
            removed[batch[q]] = 1;
            remaining--;
        }
        for (int q = 0; q < nb; q++)
            if (parent[batch[q]] >= 0) kids[parent[batch[q]]]--;
    }
    free(kids); free(removed); free(batch);
    return lev;
}

/* ------------------------- Section III.B: numeric factorisation (LDU) */

/* Row lists of a strict-lower pattern: for every row j the columns k < j with
 * (j,k) in the pattern, ascending in k, and the position of (j,k). */
static int row_lists(int n, const long long *Lp, const int *Li, long long **Rp_, int **Rk_,
                     long long **Rpos_) {
    long long nz = Lp[n];
    long long *Rp = (long long *)calloc((size_t)n + 1, sizeof(long long));
    int *Rk = (int *)malloc(sizeof(int) * (size_t)(nz > 0 ? nz : 1));
    long long *Rpos = (long long *)malloc(sizeof(long long) * (size_t)(nz > 0 ? nz : 1));
    long long *fillp = (long long *)malloc(sizeof(long long) * (size_t)(n > 0 ? n : 1));
    if (!Rp || !Rk || !Rpos || !fillp) { free(Rp); free(Rk); free(Rpos); free(fillp); return -1; }
    for (long long p = 0; p < nz; p++) Rp[Li[p] + 1]++;
    for (int j = 0; j < n; j++) Rp[j + 1] += Rp[j];
    for (int j = 0; j < n; j++) fillp[j] = Rp[j];
    for (int k = 0; k < n; k++) /* ascending k gives ascending rows lists */
        for (long long p = Lp[k]; p < Lp[k + 1]; p++) {
            long long q = fillp[Li[p]]++;
            Rk[q] = k;
            Rpos[q] = p;
        }
    free(fillp);
    *Rp_ = Rp; *Rk_ = Rk; *Rpos_ = Rpos;
    return 0;
}

/* LU without pivoting of an n x n matrix A (CSC, any order of rows within a
 * column) whose filled pattern is the symmetric pattern (Lp, Li) (strict
 * lower by column).  Left-looking with a dense work column: column j of A is
 * reduced by every earlier column k with U(k,j) != 0, in ascending k.
 * Outputs: Lx[p] = L(Li[p], k) (unit diagonal implied), Ux[p] = U(k, Li[p])
 * (the transposed position), d[k] = U(k,k).  For symmetric A, d is the D of
 * A = L D L^T and Ux = d .* Lx (Eqs. 1-3).
 * Pivot check: |d_j| <= 1e-14 max_i |A_ii| or non-finite -> OR_ERR_SINGULAR
 * (returned with *bad = j). */
int or_lu(int n, const int *Ap, const int *Ai, const double *Ax, const long long *Lp,
          const int *Li, double *Lx, double *Ux, double *d, int *bad) {
    long long *Rp = NULL, *Rpos = NULL;
    int *Rk = NULL;
    if (row_lists(n, Lp, Li, &Rp, &Rk, &Rpos)) return OR_ERR_OOM;
    double *xw = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!xw) { free(Rp); free(Rk); free(Rpos); return OR_ERR_OOM; }
    double amax = 0.0;
    for (int j = 0; j < n; j++)
        for (int p = Ap[j]; p < Ap[j + 1]; p++)
            if (Ai[p] == j && fabs(Ax[p]) > amax) amax = fabs(Ax[p]);
    int rc = OR_OK;
    if (bad) *bad = -1;
    for (int j = 0; j < n; j++) {
        for (int p = Ap[j]; p < Ap[j + 1]; p++) xw[Ai[p]] += Ax[p];
        for (long long q = Rp[j]; q < Rp[j + 1]; q++) {
            int k = Rk[q];
            double xk = xw[k];
            for (long long p = Lp[k]; p < Lp[k + 1]; p++) xw[Li[p]] -= Lx[p] * xk;
        }
        double dj = xw[j];
        d[j] = dj;
        if (!isfinite(dj) || fabs(dj) <= 1e-14 * amax) {
            rc = isfinite(dj) ? OR_ERR_SINGULAR : OR_ERR_NONFINITE;
            if (bad) *bad = j;
            break;
        }
        for (long long q = Rp[j]; q < Rp[j + 1]; q++) {
            Ux[Rpos[q]] = xw[Rk[q]];
            xw[Rk[q]] = 0.0;
        }
        for (long long p = Lp[j]; p < Lp[j + 1]; p++) {
            Lx[p] = xw[Li[p]] / dj;
            xw[Li[p]] = 0.0;
        }
        xw[j] = 0.0;
        for (int p = Ap[j]; p < Ap[j + 1]; p++) xw[Ai[p]] = 0.0;
    }
    free(xw); free(Rp); free(Rk); free(Rpos);
    return rc;
}

/* ------------------------ Section III.C: substitutions (Eq. 4 between) */

/* Solves A x = b (transpose = 0) or A^T x = b (transpose = 1) with the
 * factors of or_lu; x may alias b.
 *   A = L D Ut with Ut = D^{-1} U unit upper.
 *   forward      z_i = b_i - sum_{j<i} L_ij z_j
 *   normalise    y_i = z_i / d_ii                          (Eq. 4)
 *   backward     x_i = y_i - sum_{j>i} Ut_ij x_j
 * The transposed system uses Ut^T forward, D, and L^T backward. */
int or_lu_solve(int n, const long long *Lp, const int *Li, const double *Lx, const double *Ux,
                const double *d, const double *b, double *x, int transpose) {
    long long *Rp = NULL, *Rpos = NULL;
    int *Rk = NULL;
    if (row_lists(n, Lp, Li, &Rp, &Rk, &Rpos)) return OR_ERR_OOM;
    double *z = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!z) { free(Rp); free(Rk); free(Rpos); return OR_ERR_OOM; }
    for (int i = 0; i < n; i++) z[i] = b[i];
    /* forward: row i of the lower factor holds (i, k) for k in row list i */
    for (int i = 0; i < n; i++) {
        double s = z[i];
        for (long long q = Rp[i]; q < Rp[i + 1]; q++) {
            int k = Rk[q];
            long long p = Rpos[q];
            double lik = transpose ? Ux[p] / d[k] : Lx[p];
            s -= lik * z[k];
        }
        z[i] = s;
    }
    for (int i = 0; i < n; i++) z[i] = z[i] / d[i];
    /* backward: row k of the upper factor holds (k, i) for i in column k */
    for (int k = n - 1; k >= 0; k--) {
        double s = z[k];
        for (long long p = Lp[k]; p < Lp[k + 1]; p++) {
            double uki = transpose ? Lx[p] : Ux[p] / d[k];
            s -= uki * z[Li[p]];
        }
        z[k] = s;
    }
    for (int i = 0; i < n; i++) x[i] = z[i];
    free(z); free(Rp); free(Rk); free(Rpos);
    return OR_OK;
}

/* ------------------------------------------------------ helpers for PF */

/* A square sparse matrix on a subset of buses, permuted, with its factor. */
typedef struct {
    int n;             /* dimension */
    int *bus;          /* local -> bus (ascending bus order), length nb */
    int nb;            /* buses in the matrix */
    int *perm;         /* elimination step -> local index (length nb) */
    int *iperm;        /* local -> elimination step */
    int bs;            /* 1 scalar, 2 for the NR (theta, V) pairs */
    int *Ap, *Ai;      /* CSC of P A P^T, scalar dimension n = bs * nb */
    double *Ax;
    long long *Lp;
    int *Li;
    double *Lx, *Ux, *d;
    long long nnzL;
} fmat;

static void fmat_free(fmat *M) {
    free(M->bus); free(M->perm); free(M->iperm); free(M->Ap); free(M->Ai); free(M->Ax);
    free(M->Lp); free(M->Li); free(M->Lx); free(M->Ux); free(M->d);
    memset(M, 0, sizeof(*M));
}

/* Pattern set-up for the buses with include[bus] != 0: ordering by exact
 * minimum degree on the induced bus graph, scalar pattern of P A P^T
 * (bs x bs dense blocks), symbolic factorisation. */
static int fmat_setup(fmat *M, int n, const int *rowptr, const int *col, const char *include,
                      int bs) {
    memset(M, 0, sizeof(*M));
    M->bs = bs;
    int *loc = (int *)malloc(sizeof(int) * (size_t)n);
    if (!loc) return OR_ERR_OOM;
    int nb = 0;
    for (int i = 0; i < n; i++) loc[i] = include[i] ? nb++ : -1;
    M->nb = nb;
    M->n = bs * nb;
    M->bus = (int *)malloc(sizeof(int) * (size_t)(nb + 1));
    M->perm = (int *)malloc(sizeof(int) * (size_t)(nb + 1));
    M->iperm = (int *)malloc(sizeof(int) * (size_t)(nb + 1));
    int *gp = (int *)malloc(sizeof(int) * (size_t)(nb + 1));
    int *gi = (int *)malloc(sizeof(int) * (size_t)(rowptr[n] + 1));
    if (!M->bus || !M->perm || !M->iperm || !gp || !gi) { free(loc); free(gp); free(gi); return OR_ERR_OOM; }
    for (int i = 0; i < n; i++) if (loc[i] >= 0) M->bus[loc[i]] = i;
    /* induced local bus graph (no diagonal) */
    int nz = 0;
    gp[0] = 0;
    for (int a = 0; a < nb; a++) {
        int i = M->bus[a];
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            int j = col[p];
            if (j != i && loc[j] >= 0) gi[nz++] = loc[j];
        }
        gp[a + 1] = nz;
    }
    int rc = or_min_degree(nb, gp, gi, M->perm);
    if (rc) { free(loc); free(gp); free(gi); return rc; }
    for (int k = 0; k < nb; k++) M->iperm[M->perm[k]] = k;
    /* scalar graph of P A P^T with bs x bs blocks: vertex (step*bs + s) */
    int N = M->n;
    int *sp = (int *)malloc(sizeof(int) * (size_t)(N + 1));
    int *si = (int *)malloc(sizeof(int) * ((size_t)bs * bs * (size_t)(nz + nb) + 1));
    if (!sp || !si) { free(loc); free(gp); free(gi); free(sp); free(si); return OR_ERR_OOM; }
    int snz = 0;
    sp[0] = 0;
    for (int k = 0; k < nb; k++) {
        int a = M->perm[k];
        for (int s = 0; s < bs; s++) {
            for (int s2 = 0; s2 < bs; s2++)
                if (s2 != s) si[snz++] = k * bs + s2;
            for (int p = gp[a]; p < gp[a + 1]; p++)
                for (int s2 = 0; s2 < bs; s2++) si[snz++] = M->iperm[gi[p]] * bs + s2;
            sp[k * bs + s + 1] = snz;
        }
    }
    long long cap = 1 + (long long)N * 64;
    for (;;) {
        M->Lp = (long long *)realloc(M->Lp, sizeof(long long) * (size_t)(N + 1));
        M->Li = (int *)realloc(M->Li, sizeof(int) * (size_t)cap);
        if (!M->Lp || !M->Li) { rc = OR_ERR_OOM; break; }
        long long r = or_symbolic_etree(N, sp, si, M->Lp, M->Li, cap);
        if (r == -2) { cap *= 4; continue; }
        if (r < 0) { rc = OR_ERR_OOM; break; }
        M->nnzL = r;
        break;
    }
    free(sp); free(si); free(loc); free(gp); free(gi);
    if (rc) return rc;
    M->Lx = (double *)malloc(sizeof(double) * (size_t)(M->nnzL + 1));
    M->Ux = (double *)malloc(sizeof(double) * (size_t)(M->nnzL + 1));
    M->d = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    if (!M->Lx || !M->Ux || !M->d) return OR_ERR_OOM;
    return OR_OK;
}

/* Scalar B-type matrix (B' or B'') of the included buses from values on the
 * Ybus pattern, as CSC of P A P^T. */
static int fmat_values_scalar(fmat *M, int n, const int *rowptr, const int *col, const double *V,
                              double scale) {
    int N = M->n;
    int *loc = (int *)malloc(sizeof(int) * (size_t)n);
    if (!loc) return OR_ERR_OOM;
    for (int i = 0; i < n; i++) loc[i] = -1;
    for (int a = 0; a < M->nb; a++) loc[M->bus[a]] = a;
    free(M->Ap); free(M->Ai); free(M->Ax);
    M->Ap = (int *)calloc((size_t)N + 1, sizeof(int));
    int cnt = 0;
    for (int a = 0; a < M->nb; a++) {
        int i = M->bus[a];
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (loc[col[p]] >= 0) cnt++;
    }
    M->Ai = (int *)malloc(sizeof(int) * (size_t)(cnt + 1));
    M->Ax = (double *)malloc(sizeof(double) * (size_t)(cnt + 1));
    if (!M->Ap || !M->Ai || !M->Ax) { free(loc); return OR_ERR_OOM; }
    /* column c of P A P^T = row/column bus[perm[c]] of the symmetric-pattern A;
     * A is stored by rows, so column j of A is read as row j of A^T: for B'
     * and B'' (symmetric) the two coincide. */
    int q = 0;
    for (int c = 0; c < N; c++) {
        int i = M->bus[M->perm[c]];
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++) {
            int j = col[p];
            if (loc[j] < 0) continue;
            /* entry (row = j, col = i) of A; A symmetric so A(j,i) = A(i,j) */
            M->Ai[q] = M->iperm[loc[j]];
            M->Ax[q] = scale * V[p];
            q++;
        }
        M->Ap[c + 1] = q;
    }
    free(loc);
    return OR_OK;
}

/* Polar Newton-Raphson Jacobian on the non-slack buses, CSC of P J P^T with
 * unknown pair (theta, V) per bus.  Row pair (P_i, Q_i); PV buses have their
 * Q row and V column replaced by the identity.  Needs P, Q at the state. */
static int fmat_values_jacobian(fmat *M, int n, const int *btype, const int *rowptr,
                                const int *col, const double *G, const double *B,
                                const double *vm, const double *va, const double *P,
                                const double *Q) {
    int N = M->n;
    int *loc = (int *)malloc(sizeof(int) * (size_t)n);
    if (!loc) return OR_ERR_OOM;
    for (int i = 0; i < n; i++) loc[i] = -1;
    for (int a = 0; a < M->nb; a++) loc[M->bus[a]] = a;
    free(M->Ap); free(M->Ai); free(M->Ax);
    int cnt = 0;
    for (int a = 0; a < M->nb; a++) {
        int i = M->bus[a];
        for (int p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (loc[col[p]] >= 0) cnt++;
    }
    M->Ap = (int *)calloc((size_t)N + 1, sizeof(int));
    M->Ai = (int *)malloc(sizeof(int) * (size_t)(4 * cnt + 1));
    M->Ax = (double *)malloc(sizeof(double) * (size_t)(4 * cnt + 1));
    if (!M->Ap || !M->Ai || !M->Ax) { free(loc); return OR_ERR_OOM; }
    int q = 0;
    /* column pair of bus k = bus[perm[c]]: entries in rows of buses i adjacent to k.
     * The pattern is symmetric, so the rows of column k are the columns of row k. */
    for (int c = 0; c < M->nb; c++) {
        int k = M->bus[M->perm[c]];
        for (int s = 0; s < 2; s++) { /* s = 0: d/dtheta_k, s = 1: d/dV_k */
            for (int p = rowptr[k]; p < rowptr[k + 1]; p++) {
                int i = col[p];
                if (loc[i] < 0) continue;
                int pik = csr_pos(rowptr, col, i, k); /* Y_ik */
                double g = G[pik], bb = B[pik];
                double th = va[i] - va[k];
                double cs = cos(th), sn = sin(th);
                double dP, dQ;
                if (i != k) {
                    if (s == 0) {
                        dP = vm[i] * vm[k] * (g * sn - bb * cs);
                        dQ = -vm[i] * vm[k] * (g * cs + bb * sn);
                    } else {
                        dP = vm[i] * (g * cs + bb * sn);
                        dQ = vm[i] * (g * sn - bb * cs);
                    }
                } else {
                    if (s == 0) {
                        dP = -Q[i] - bb * vm[i] * vm[i];
                        dQ = P[i] - g * vm[i] * vm[i];
                    } else {
                        dP = P[i] / vm[i] + g * vm[i];
                        dQ = Q[i] / vm[i] - bb * vm[i];
                    }
                }
                int ri = M->iperm[loc[i]] * 2;
                if (s == 1 && btype[k] == OR_PV) { /* pinned V column */
                    dP = 0.0;
                    dQ = (i == k) ? 1.0 : 0.0;
                }
                if (btype[i] == OR_PV) /* Q row of a PV bus is the identity row */
                    dQ = (i == k && s == 1) ? 1.0 : 0.0;
                M->Ai[q] = ri; M->Ax[q] = dP; q++;
                M->Ai[q] = ri + 1; M->Ax[q] = dQ; q++;
            }
            M->Ap[2 * c + s + 1] = q;
        }
    }
    free(loc);
    return OR_OK;
}

static int fmat_factor(fmat *M) {
    int bad;
    return or_lu(M->n, M->Ap, M->Ai, M->Ax, M->Lp, M->Li, M->Lx, M->Ux, M->d, &bad);
}

/* Export helpers for tests: the pieces of the factored NR/B matrices. */

/* ------------------------------------------ Section III: power flow */

/* Full power flow from the bus/branch tables.
 *   method: OR_FDPF (XB fast decoupled) or OR_NR (polar Newton-Raphson).
 *   start_from_input: 0 -> flat start (theta = 0, V = 1 at PQ, vset at PV
 *   and slack, slack angle va0); 1 -> start from vm/va as given.
 *   On return vm/va hold the final state, *iters the number of linear solves
 *   taken (NR steps, or FDPF half-iterations), *maxmis the last mismatch.
 * Returns OR_OK, OR_ERR_NOT_CONVERGED, OR_ERR_SINGULAR, OR_ERR_NONFINITE,
 * OR_ERR_ARG or OR_ERR_OOM. */
int or_power_flow(int method, int n, int m, const int *btype, const double *pd, const double *qd,
                  const double *gs, const double *bs, const double *pg, const double *vset,
                  const double *va0, const int *f, const int *t, const double *r,
                  const double *x, const double *b, const double *tap, const int *status,
                  double tol, int max_iter, int start_from_input, double *vm, double *va,
                  int *iters, double *maxmis) {
    int rc = OR_OK;
    int *rowptr = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    int *col = (int *)malloc(sizeof(int) * (size_t)(n + 2 * m + 1));
    double *G = NULL, *B = NULL, *Bp = NULL, *Bpp = NULL, *Psp = NULL, *Qsp = NULL, *P = NULL,
           *Q = NULL, *dP = NULL, *dQ = NULL, *rhs = NULL;
    char *inc = NULL;
    fmat M1, M2;
    memset(&M1, 0, sizeof(M1));
    memset(&M2, 0, sizeof(M2));
    *iters = 0;
    *maxmis = INFINITY;
    if (!rowptr || !col) { rc = OR_ERR_OOM; goto out; }
    for (int i = 0; i < n; i++)
        if (btype[i] < OR_PQ || btype[i] > OR_SLACK) { rc = OR_ERR_ARG; goto out; }
    int nnz = or_ybus_pattern(n, m, f, t, rowptr, col);
    if (nnz < 0) { rc = OR_ERR_ARG; goto out; }
    G = (double *)malloc(sizeof(double) * (size_t)nnz);
    B = (double *)malloc(sizeof(double) * (size_t)nnz);
    Bp = (double *)malloc(sizeof(double) * (size_t)nnz);
    Bpp = (double *)malloc(sizeof(double) * (size_t)nnz);
    Psp = (double *)malloc(sizeof(double) * (size_t)n);
    Qsp = (double *)malloc(sizeof(double) * (size_t)n);
    P = (double *)malloc(sizeof(double) * (size_t)n);
    Q = (double *)malloc(sizeof(double) * (size_t)n);
    dP = (double *)malloc(sizeof(double) * (size_t)n);
    dQ = (double *)malloc(sizeof(double) * (size_t)n);
    rhs = (double *)malloc(sizeof(double) * (size_t)(2 * n + 2));
    inc = (char *)malloc((size_t)n + 1);
    if (!G || !B || !Bp || !Bpp || !Psp || !Qsp || !P || !Q || !dP || !dQ || !rhs || !inc) {
        rc = OR_ERR_OOM;
        goto out;
    }
    rc = or_ybus_values(n, m, f, t, r, x, b, tap, status, gs, bs, rowptr, col, G, B);
    if (rc) goto out;
    for (int i = 0; i < n; i++) {
        Psp[i] = pg[i] - pd[i];
        Qsp[i] = -qd[i];
        if (!start_from_input) {
            vm[i] = (btype[i] == OR_PQ) ? 1.0 : vset[i];
            va[i] = (btype[i] == OR_SLACK) ? va0[i] : 0.0;
        }
    }
    if (method == OR_FDPF) {
        rc = or_bprime_values(n, m, f, t, x, status, rowptr, col, Bp);
        if (rc) goto out;
        for (int p = 0; p < nnz; p++) Bpp[p] = -B[p];
        for (int i = 0; i < n; i++) inc[i] = btype[i] != OR_SLACK;
        if ((rc = fmat_setup(&M1, n, rowptr, col, inc, 1))) goto out;
        for (int i = 0; i < n; i++) inc[i] = btype[i] == OR_PQ;
        if ((rc = fmat_setup(&M2, n, rowptr, col, inc, 1))) goto out;
        if ((rc = fmat_values_scalar(&M1, n, rowptr, col, Bp, 1.0))) goto out;
        if ((rc = fmat_values_scalar(&M2, n, rowptr, col, Bpp, 1.0))) goto out;
        if ((rc = fmat_factor(&M1))) goto out;
        if ((rc = fmat_factor(&M2))) goto out;
        rc = OR_ERR_NOT_CONVERGED;
        for (int it = 0; it < max_iter; it++) {
            /* P half-iteration: B' dtheta = dP / V */
            or_injections(n, rowptr, col, G, B, vm, va, P, Q);
            *maxmis = or_mismatch(n, btype, Psp, Qsp, P, Q, dP, dQ);
            if (!isfinite(*maxmis)) { rc = OR_ERR_NONFINITE; break; }
            if (*maxmis <= tol) { rc = OR_OK; break; }
            for (int c = 0; c < M1.n; c++) { int i = M1.bus[M1.perm[c]]; rhs[c] = dP[i] / vm[i]; }
            or_lu_solve(M1.n, M1.Lp, M1.Li, M1.Lx, M1.Ux, M1.d, rhs, rhs, 0);
            for (int c = 0; c < M1.n; c++) va[M1.bus[M1.perm[c]]] += rhs[c];
            (*iters)++;
            /* Q half-iteration: B'' dV = dQ / V */
            or_injections(n, rowptr, col, G, B, vm, va, P, Q);
            *maxmis = or_mismatch(n, btype, Psp, Qsp, P, Q, dP, dQ);
            if (!isfinite(*maxmis)) { rc = OR_ERR_NONFINITE; break; }
            if (*maxmis <= tol) { rc = OR_OK; break; }
            for (int c = 0; c < M2.n; c++) { int i = M2.bus[M2.perm[c]]; rhs[c] = dQ[i] / vm[i]; }
            or_lu_solve(M2.n, M2.Lp, M2.Li, M2.Lx, M2.Ux, M2.d, rhs, rhs, 0);
            for (int c = 0; c < M2.n; c++) vm[M2.bus[M2.perm[c]]] += rhs[c];
            (*iters)++;
        }
        if (rc == OR_ERR_NOT_CONVERGED) { /* final check after the last pair */
            or_injections(n, rowptr, col, G, B, vm, va, P, Q);
            *maxmis = or_mismatch(n, btype, Psp, Qsp, P, Q, dP, dQ);
            if (*maxmis <= tol) rc = OR_OK;
        }
    } else if (method == OR_NR) {
        for (int i = 0; i < n; i++) inc[i] = btype[i] != OR_SLACK;
        if ((rc = fmat_setup(&M1, n, rowptr, col, inc, 2))) goto out;
        rc = OR_ERR_NOT_CONVERGED;
        for (int it = 0; it <= max_iter; it++) {
            or_injections(n, rowptr, col, G, B, vm, va, P, Q);
            *maxmis = or_mismatch(n, btype, Psp, Qsp, P, Q, dP, dQ);
            if (!isfinite(*maxmis)) { rc = OR_ERR_NONFINITE; break; }
            if (*maxmis <= tol) { rc = OR_OK; break; }
            if (it == max_iter) break;
            int frc = fmat_values_jacobian(&M1, n, btype, rowptr, col, G, B, vm, va, P, Q);
            if (frc) { rc = frc; break; }
            if ((frc = fmat_factor(&M1))) { rc = frc; break; }
            for (int c = 0; c < M1.nb; c++) {
                int i = M1.bus[M1.perm[c]];
                rhs[2 * c] = dP[i];
                rhs[2 * c + 1] = (btype[i] == OR_PQ) ? dQ[i] : 0.0;
            }
            or_lu_solve(M1.n, M1.Lp, M1.Li, M1.Lx, M1.Ux, M1.d, rhs, rhs, 0);
            for (int c = 0; c < M1.nb; c++) {
                int i = M1.bus[M1.perm[c]];
                va[i] += rhs[2 * c];
                if (btype[i] == OR_PQ) vm[i] += rhs[2 * c + 1];
            }
            (*iters)++;
        }
    } else {
        rc = OR_ERR_ARG;
    }
out:
    fmat_free(&M1);
    fmat_free(&M2);
    free(rowptr); free(col); free(G); free(B); free(Bp); free(Bpp); free(Psp); free(Qsp);
    free(P); free(Q); free(dP); free(dQ); free(rhs); free(inc);
    return rc;
}

/* ------------------------------------------ adjoint of the power flow */

/* Objective J(x) = sum_i (V_i - 1)^2 + sum_i P_i(V, theta) over all buses
 * (the second sum is the total active loss).  With F(x) = Psp - P(x) on the
 * Newton-Raphson rows, dJ/dPsp = lambda where J_x(x*)^T lambda = grad_x J.
 * The Jacobian is factorised afresh at the given state x*.
 * Outputs dJdP[i] (non-slack, else 0), dJdQ[i] (PQ, else 0) and *Jval. */
int or_adjoint(int n, int m, const int *btype, const double *gs, const double *bs,
               const int *f, const int *t, const double *r, const double *x, const double *b,
               const double *tap, const int *status, const double *vm, const double *va,
               double *dJdP, double *dJdQ, double *Jval) {
    int rc = OR_OK;
    int *rowptr = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    int *col = (int *)malloc(sizeof(int) * (size_t)(n + 2 * m + 1));
    double *G = NULL, *B = NULL, *P = NULL, *Q = NULL, *gth = NULL, *gv = NULL, *rhs = NULL;
    char *inc = NULL;
    fmat M;
    memset(&M, 0, sizeof(M));
    if (!rowptr || !col) { rc = OR_ERR_OOM; goto out; }
    int nnz = or_ybus_pattern(n, m, f, t, rowptr, col);
    if (nnz < 0) { rc = OR_ERR_ARG; goto out; }
    G = (double *)malloc(sizeof(double) * (size_t)nnz);
    B = (double *)malloc(sizeof(double) * (size_t)nnz);
    P = (double *)malloc(sizeof(double) * (size_t)n);
    Q = (double *)malloc(sizeof(double) * (size_t)n);
    gth = (double *)calloc((size_t)n, sizeof(double));
    gv = (double *)calloc((size_t)n, sizeof(double));
    rhs = (double *)malloc(sizeof(double) * (size_t)(2 * n + 2));
    inc = (char *)malloc((size_t)n + 1);
    if (!G || !B || !P || !Q || !gth || !gv || !rhs || !inc) { rc = OR_ERR_OOM; goto out; }
    if ((rc = or_ybus_values(n, m, f, t, r, x, b, tap, status, gs, bs, rowptr, col, G, B))) goto out;
    or_injections(n, rowptr, col, G, B, vm, va, P, Q);
    double J = 0.0;
    for (int i = 0; i < n; i++) J += (vm[i] - 1.0) * (vm[i] - 1.0) + P[i];
    *Jval = J;
    /* grad of sum_l P_l: column sums of dP_l/dtheta_k and dP_l/dV_k over every row l */
    for (int l = 0; l < n; l++)
        for (int p = rowptr[l]; p < rowptr[l + 1]; p++) {
            int k = col[p];
            double g = G[p], bb = B[p];
            double th = va[l] - va[k], cs = cos(th), sn = sin(th);
            if (k != l) {
                gth[k] += vm[l] * vm[k] * (g * sn - bb * cs);
                gv[k] += vm[l] * (g * cs + bb * sn);
            } else {
                gth[k] += -Q[l] - bb * vm[l] * vm[l];
                gv[k] += P[l] / vm[l] + g * vm[l];
            }
        }
    for (int i = 0; i < n; i++) gv[i] += 2.0 * (vm[i] - 1.0);
    for (int i = 0; i < n; i++) inc[i] = btype[i] != OR_SLACK;
    if ((rc = fmat_setup(&M, n, rowptr, col, inc, 2))) goto out;
    if ((rc = fmat_values_jacobian(&M, n, btype, rowptr, col, G, B, vm, va, P, Q))) goto out;
    if ((rc = fmat_factor(&M))) goto out;
    for (int c = 0; c < M.nb; c++) {
        int i = M.bus[M.perm[c]];
        rhs[2 * c] = gth[i];
        rhs[2 * c + 1] = (btype[i] == OR_PQ) ? gv[i] : 0.0;
    }
    if ((rc = or_lu_solve(M.n, M.Lp, M.Li, M.Lx, M.Ux, M.d, rhs, rhs, 1))) goto out;
    for (int i = 0; i < n; i++) { dJdP[i] = 0.0; dJdQ[i] = 0.0; }
    for (int c = 0; c < M.nb; c++) {
        int i = M.bus[M.perm[c]];
        dJdP[i] = rhs[2 * c];
        dJdQ[i] = (btype[i] == OR_PQ) ? rhs[2 * c + 1] : 0.0;
    }
out:
    fmat_free(&M);
    free(rowptr); free(col); free(G); free(B); free(P); free(Q); free(gth); free(gv);
    free(rhs); free(inc);
    return rc;
}

/* Dense export of the NR Jacobian at a state (tests compare it with finite
 * differences of or_injections).  Row/column order: natural non-slack bus
 * order, pair (theta, V) per bus.  J must hold (2 nb)^2 doubles where nb is
 * the number of non-slack buses. */
int or_jacobian_dense(int n, int m, const int *btype, const double *gs, const double *bs,
                      const int *f, const int *t, const double *r, const double *x,
                      const double *b, const double *tap, const int *status, const double *vm,
                      const double *va, double *Jd) {
    int rc = OR_OK;
    int *rowptr = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    int *col = (int *)malloc(sizeof(int) * (size_t)(n + 2 * m + 1));
    double *G = NULL, *B = NULL, *P = NULL, *Q = NULL;
    char *inc = (char *)malloc((size_t)n + 1);
    fmat M;
    memset(&M, 0, sizeof(M));
    int nnz = or_ybus_pattern(n, m, f, t, rowptr, col);
    if (nnz < 0) { rc = OR_ERR_ARG; goto out; }
    G = (double *)malloc(sizeof(double) * (size_t)nnz);
    B = (double *)malloc(sizeof(double) * (size_t)nnz);
    P = (double *)malloc(sizeof(double) * (size_t)n);
    Q = (double *)malloc(sizeof(double) * (size_t)n);
    if ((rc = or_ybus_values(n, m, f, t, r, x, b, tap, status, gs, bs, rowptr, col, G, B))) goto out;
    or_injections(n, rowptr, col, G, B, vm, va, P, Q);
    for (int i = 0; i < n; i++) inc[i] = btype[i] != OR_SLACK;
    if ((rc = fmat_setup(&M, n, rowptr, col, inc, 2))) goto out;
    if ((rc = fmat_values_jacobian(&M, n, btype, rowptr, col, G, B, vm, va, P, Q))) goto out;
    {
        int N = M.n;
        for (long long z = 0; z < (long long)N * N; z++) Jd[z] = 0.0;
        for (int c = 0; c < N; c++) {
            int cb = M.perm[c / 2] * 2 + (c % 2);
            for (int p = M.Ap[c]; p < M.Ap[c + 1]; p++) {
                int rr = M.Ai[p];
                int rb = M.perm[rr / 2] * 2 + (rr % 2);
                Jd[(long long)rb * N + cb] += M.Ax[p];
            }
        }
    }
out:
    fmat_free(&M);
    free(rowptr); free(col); free(G); free(B); free(P); free(Q); free(inc);
    return rc;
}
