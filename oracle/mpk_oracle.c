/*
 * FP64 CPU oracle for the level-blocked matrix-power kernel (MPK).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header or table with the CUDA
 * library.  Every routine is a plain sequential restatement of a definition
 * of the paper (Alappat et al., "Level-based Blocking for Sparse Matrices:
 * Sparse Matrix-Power-Vector Multiplication"), cited per routine.
 *
 * Compiled with -O2 -ffp-contract=off so that every product and sum is a
 * separately rounded IEEE binary64 operation, in the stored column order.
 *
 * Matrices are CRS with int32 row pointers and column indices (Sec. 3.1,
 * Fig. 1).  Block vectors are row-major n x nrhs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

int oracle_abi_version(void) { return 1; }

/* ------------------------------------------------------------------ SpMV
 * Fig. 1 (Sec. 3.1): out[row] = sum over the stored entries of `row` of
 * val[idx] * in[col[idx]], for rows row_s..row_e inclusive, in stored order.
 */
void oracle_spmv_rows(const int32_t *rowptr, const int32_t *col, const double *val,
                      int32_t nrhs, const double *in, double *out,
                      int32_t row_s, int32_t row_e)
{
    for (int32_t row = row_s; row <= row_e; row++) {
        for (int32_t c = 0; c < nrhs; c++) {
            double tmp = 0.0;
            for (int32_t idx = rowptr[row]; idx < rowptr[row + 1]; idx++)
                tmp += val[idx] * in[(int64_t)col[idx] * nrhs + c];
            out[(int64_t)row * nrhs + c] = tmp;
        }
    }
}

/* Baseline MPK (Sec. 3.1, Fig. 1): y_0 = x, y_p = A y_{p-1} for p = 1..pm.
 * Y holds pm blocks of n*nrhs doubles, block p-1 = y_p. */
void oracle_mpk(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                int32_t pm, int32_t nrhs, const double *x, double *Y)
{
    const int64_t blk = (int64_t)n * nrhs;
    for (int32_t p = 1; p <= pm; p++) {
        const double *in = (p == 1) ? x : Y + (int64_t)(p - 2) * blk;
        if (n > 0)
            oracle_spmv_rows(rowptr, col, val, nrhs, in, Y + (int64_t)(p - 1) * blk, 0, n - 1);
    }
}

/* ------------------------------------------------------------------ levels
 * Eq. 3 (Sec. 4.1): L(0) = {root}; L(i) = vertices in the neighbourhood of
 * L(i-1) that carry no level yet.  Computed with a FIFO breadth-first search:
 * a vertex's level is its hop distance from the root.
 *
 * Readings where the paper is silent:
 *  - neighbourhood = stored pattern of A, plus that of A^T when `symmetrize`
 *    is set (the paper restricts itself to symmetric patterns, Sec. 4);
 *  - when the queue empties while vertices remain unvisited (a disconnected
 *    graph), the lowest-numbered unvisited vertex starts a new component at
 *    the next level number.
 * Returns the number of levels L_m; level[v] receives v's level.
 */
int32_t oracle_bfs_levels(int32_t n, const int32_t *rowptr, const int32_t *col,
                          int32_t root, int32_t symmetrize, int32_t *level)
{
    if (n <= 0) return 0;
    int32_t *trp = NULL, *tcol = NULL;
    if (symmetrize) {             /* CRS of the transposed pattern */
        int64_t nnz = rowptr[n];
        trp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        tcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
        for (int64_t e = 0; e < nnz; e++) trp[col[e] + 1]++;
        for (int32_t v = 0; v < n; v++) trp[v + 1] += trp[v];
        int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        memcpy(fill, trp, sizeof(int32_t) * (size_t)n);
        for (int32_t u = 0; u < n; u++)
            for (int32_t e = rowptr[u]; e < rowptr[u + 1]; e++) tcol[fill[col[e]]++] = u;
        free(fill);
    }
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int32_t v = 0; v < n; v++) level[v] = -1;
    int32_t head = 0, tail = 0, maxlevel = -1, next_unvisited = 0;
    int32_t start = (root >= 0 && root < n) ? root : 0;
    for (;;) {
        level[start] = maxlevel + 1;
        queue[tail++] = start;
        while (head < tail) {
            int32_t u = queue[head++];
            if (level[u] > maxlevel) maxlevel = level[u];
            for (int32_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
                int32_t v = col[e];
                if (level[v] < 0) { level[v] = level[u] + 1; queue[tail++] = v; }
            }
            if (symmetrize)
                for (int32_t e = trp[u]; e < trp[u + 1]; e++) {
                    int32_t v = tcol[e];
                    if (level[v] < 0) { level[v] = level[u] + 1; queue[tail++] = v; }
                }
        }
        while (next_unvisited < n && level[next_unvisited] >= 0) next_unvisited++;
        if (next_unvisited == n) break;
        start = next_unvisited;
    }
    free(queue); free(trp); free(tcol);
    return maxlevel + 1;
}

/* Sec. 4.1: renumber so that the vertices of L(i-1) precede those of L(i)
 * and each level is consecutive.  Reading: inside a level, ascending
 * original index (a stable counting sort by level).
 * perm[new] = old, iperm[old] = new, level_ptr[i] = first new index of L(i)
 * (Fig. 3e), level_ptr[nlevels] = n. */
void oracle_level_perm(int32_t n, const int32_t *level, int32_t nlevels,
                       int32_t *perm, int32_t *iperm, int32_t *level_ptr)
{
    for (int32_t i = 0; i <= nlevels; i++) level_ptr[i] = 0;
    for (int32_t v = 0; v < n; v++) level_ptr[level[v] + 1]++;
    for (int32_t i = 0; i < nlevels; i++) level_ptr[i + 1] += level_ptr[i];
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nlevels > 0 ? nlevels : 1));
    for (int32_t i = 0; i < nlevels; i++) pos[i] = level_ptr[i];
    for (int32_t v = 0; v < n; v++) {
        int32_t r = pos[level[v]]++;
        perm[r] = v;
        iperm[v] = r;
    }
    free(pos);
}

/* Symmetric permutation P A P^T (Sec. 4.1 footnote): new row r is old row
 * perm[r], each column c becomes iperm[c]; entries of a row are put in
 * ascending new-column order (stable for equal columns).  Output arrays
 * are caller-allocated with n+1 / nnz entries. */
void oracle_permute_csr(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                        const int32_t *perm, const int32_t *iperm,
                        int32_t *prow, int32_t *pcol, double *pval)
{
    prow[0] = 0;
    for (int32_t r = 0; r < n; r++) {
        int32_t o = perm[r];
        int32_t len = rowptr[o + 1] - rowptr[o];
        int32_t base = prow[r];
        prow[r + 1] = base + len;
        for (int32_t j = 0; j < len; j++) {            /* insertion sort */
            int32_t c = iperm[col[rowptr[o] + j]];
            double a = val[rowptr[o] + j];
            int32_t k = base + j;
            while (k > base && pcol[k - 1] > c) { pcol[k] = pcol[k - 1]; pval[k] = pval[k - 1]; k--; }
            pcol[k] = c; pval[k] = a;
        }
    }
}

/* ------------------------------------------------------------------ groups
 * Eq. 5 (Sec. 4.2.1): starting at the first level not yet grouped, add
 * consecutive levels to the group while (pm+1) * weight(T) < f * C holds,
 * where weight(T) is the sum of the member levels' weights (the paper uses
 * Nnz(T) * 12 bytes).  A level that violates the bound on its own forms a
 * group by itself.  group_ptr[g] = first level of T(g); returns the group
 * count G (group_ptr[G] = nlevels). */
int32_t oracle_level_groups(int32_t nlevels, const double *level_weight, int32_t pm,
                            double f, double C, int32_t *group_ptr)
{
    int32_t G = 0, start = 0;
    const double budget = f * C;
    while (start < nlevels) {
        double acc = level_weight[start];
        int32_t end = start + 1;
        while (end < nlevels && (double)(pm + 1) * (acc + level_weight[end]) < budget) {
            acc += level_weight[end];
            end++;
        }
        group_ptr[G++] = start;
        start = end;
    }
    group_ptr[G] = nlevels;
    return G;
}

/* ------------------------------------------------------------------ recursion
 * Sec. 4.4: levels and level groups refined recursively inside bulky groups.
 *
 * Stage 0 is Sec. 4.1-4.2: the Eq. 3 levels (oracle_bfs_levels, root
 * `root`), the level-consecutive renumbering (oracle_level_perm) and the
 * greedy groups of Eq. 5 (oracle_level_groups) over the level weights, a
 * level's weight being the sum of w[v] over its vertices.  A group is bulky
 * when it violates Eq. 5: it holds a single level and (pm+1)*weight >= f*C.
 * Then, for stages s = 0 .. s_max-1, every maximal run of consecutive bulky
 * groups is refined:
 *   - the subgraph induced by the run's vertices (edges of the stored
 *     pattern between two vertices of the run) gets its own BFS levels by
 *     Eq. 3, rooted at the run's first vertex in the current numbering; when
 *     the search runs out, the run's lowest-numbered (current numbering)
 *     unvisited vertex starts the next level (the restart rule of the
 *     stage-0 levels);
 *   - the run's vertices are renumbered by (sub-level, current number), in
 *     place of the run;
 *   - the run's groups are replaced by the Eq. 5 groups of its sub-levels,
 *     which belong to stage s+1; bulky ones among them are refined at the
 *     next stage.
 * Readings where the paper is silent: the root of a subgraph's search and
 * the restart rule inside it; "consecutive" bulky groups form one subgraph.
 *
 * Outputs (caller-allocated, size n or n+1): perm[new] = old; the finest
 * levels level_ptr[0..*nlevels] (first new vertex of each; level_ptr[*nlevels]
 * = n); the groups group_ptr[0..*ngroups] as ranges of those levels; and
 * group_stage[g], the recursion stage that made group g.  The pattern must
 * be structurally symmetric.  Returns the number of stages that refined
 * something (0 .. s_max).
 */
static int32_t groups_of_levels(int32_t l0, int32_t l1, const double *lw, int32_t pm, double f, double C,
                                int32_t *gp_out)
{   /* Eq. 5 over levels l0..l1-1; group starts (absolute level indices) */
    return oracle_level_groups(l1 - l0, lw + l0, pm, f, C, gp_out);
}

int32_t oracle_recursive_levels(int32_t n, const int32_t *rowptr, const int32_t *col, int32_t root,
                                const double *w, int32_t pm, double f, double C, int32_t s_max,
                                int32_t *perm, int32_t *level_ptr, int32_t *nlevels,
                                int32_t *group_ptr, int32_t *ngroups, int32_t *group_stage)
{
    int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *iperm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t L = oracle_bfs_levels(n, rowptr, col, root, 0, level);
    /* current state: perm / iperm, flat levels lp[0..L], groups gp[0..G] with stages gs[] */
    int32_t *lp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    oracle_level_perm(n, level, L, perm, iperm, lp);
    double *lw = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    int32_t *gp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *gs = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    for (int32_t l = 0; l < L; l++) {
        lw[l] = 0.0;
        for (int32_t r = lp[l]; r < lp[l + 1]; r++) lw[l] += w[perm[r]];
    }
    int32_t G = oracle_level_groups(L, lw, pm, f, C, gp);
    for (int32_t g = 0; g < G; g++) gs[g] = 0;

    /* scratch for the next state */
    int32_t *lp2 = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *gp2 = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *gs2 = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    double *lw2 = (double *)malloc(sizeof(double) * ((size_t)n + 1));
    int32_t *perm2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *sub = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);      /* sub-level per run position */
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    const double budget = f * C;
    int32_t stages = 0;

    for (int32_t s = 0; s < s_max; s++) {
        int32_t L2 = 0, G2 = 0, refined = 0;
        memcpy(perm2, perm, sizeof(int32_t) * (size_t)n);
        int32_t g = 0;
        while (g < G) {
            const int bulky = gp[g + 1] - gp[g] == 1 && (double)(pm + 1) * lw[gp[g]] >= budget;
            if (!bulky) {   /* copy the group and its levels unchanged */
                gp2[G2] = L2;
                gs2[G2++] = gs[g];
                for (int32_t l = gp[g]; l < gp[g + 1]; l++) {
                    lp2[L2] = lp[l];
                    lw2[L2++] = lw[l];
                }
                g++;
                continue;
            }
            int32_t g1 = g;   /* maximal run of bulky groups g .. g1-1 */
            while (g1 < G && gp[g1 + 1] - gp[g1] == 1 && (double)(pm + 1) * lw[gp[g1]] >= budget) g1++;
            const int32_t a = lp[gp[g]], b = lp[gp[g1]], m = b - a;
            /* Eq. 3 on the induced subgraph of rows a..b-1 (current numbering) */
            for (int32_t i = 0; i < m; i++) sub[i] = -1;
            int32_t head = 0, tail = 0, maxlev = -1, next = 0, start = 0;
            for (;;) {
                sub[start] = maxlev + 1;
                queue[tail++] = start;
                while (head < tail) {
                    const int32_t u = queue[head++];
                    if (sub[u] > maxlev) maxlev = sub[u];
                    const int32_t ou = perm[a + u];
                    for (int32_t e = rowptr[ou]; e < rowptr[ou + 1]; e++) {
                        const int32_t v = iperm[col[e]] - a;
                        if (v >= 0 && v < m && sub[v] < 0) { sub[v] = sub[u] + 1; queue[tail++] = v; }
                    }
                }
                while (next < m && sub[next] >= 0) next++;
                if (next == m) break;
                start = next;
            }
            const int32_t Ls = maxlev + 1;
            /* renumber by (sub-level, current number): stable counting sort */
            for (int32_t l = 0; l <= Ls; l++) tmp[l] = 0;
            for (int32_t i = 0; i < m; i++) tmp[sub[i] + 1]++;
            for (int32_t l = 0; l < Ls; l++) tmp[l + 1] += tmp[l];
            const int32_t lbase = L2;
            for (int32_t l = 0; l < Ls; l++) {
                lp2[L2 + l] = a + tmp[l];
                lw2[L2 + l] = 0.0;
            }
            for (int32_t i = 0; i < m; i++) {
                const int32_t r = a + tmp[sub[i]]++;
                perm2[r] = perm[a + i];
                lw2[L2 + sub[i]] += w[perm[a + i]];
            }
            L2 += Ls;
            /* Eq. 5 groups of the sub-levels, stage s+1 */
            const int32_t Gs = groups_of_levels(lbase, L2, lw2, pm, f, C, tmp);
            for (int32_t q = 0; q < Gs; q++) {
                gp2[G2] = lbase + tmp[q];
                gs2[G2++] = s + 1;
            }
            refined = 1;
            g = g1;
        }
        lp2[L2] = n;
        gp2[G2] = L2;
        if (!refined) break;
        stages = s + 1;
        memcpy(perm, perm2, sizeof(int32_t) * (size_t)n);
        for (int32_t r = 0; r < n; r++) iperm[perm[r]] = r;
        memcpy(lp, lp2, sizeof(int32_t) * ((size_t)L2 + 1));
        memcpy(lw, lw2, sizeof(double) * (size_t)L2);
        memcpy(gp, gp2, sizeof(int32_t) * ((size_t)G2 + 1));
        memcpy(gs, gs2, sizeof(int32_t) * (size_t)G2);
        L = L2;
        G = G2;
    }
    memcpy(level_ptr, lp, sizeof(int32_t) * ((size_t)L + 1));
    memcpy(group_ptr, gp, sizeof(int32_t) * ((size_t)G + 1));
    memcpy(group_stage, gs, sizeof(int32_t) * (size_t)G);
    *nlevels = L;
    *ngroups = G;
    free(level); free(iperm); free(lp); free(lw); free(gp); free(gs); free(lp2); free(gp2); free(gs2);
    free(lw2); free(perm2); free(sub); free(queue); free(tmp);
    return stages;
}

/* ------------------------------------------------------------------ Lp order
 * Fig. 5 (Sec. 4.2): diagonals d = i + p ascending from 1 to L_m + pm - 1;
 * inside a diagonal, p ascending from max(1, d - L_m + 1) to min(d, pm);
 * node (i, p) with i = d - p.  Writes the nodes in execution order (step 0
 * first) into node_i / node_p; returns the number of nodes (L_m * pm). */
int64_t oracle_lp_order(int32_t nlevels, int32_t pm, int32_t *node_i, int32_t *node_p)
{
    int64_t s = 0;
    for (int32_t d = 1; d <= nlevels + pm - 1; d++) {
        int32_t p_start = (d - nlevels + 1 > 1) ? d - nlevels + 1 : 1;
        int32_t p_end = (d < pm) ? d : pm;
        for (int32_t p = p_start; p <= p_end; p++) {
            node_i[s] = d - p;
            node_p[s] = p;
            s++;
        }
    }
    return s;
}

/* Level-blocked MPK (Fig. 5) run sequentially on an already permuted
 * matrix: every node (i, p) applies the SpMV of Fig. 1 to the rows of unit i
 * (unit_ptr[i] .. unit_ptr[i+1]-1) reading y_{p-1}.  With unit_ptr =
 * level_ptr this is the basic LB MPK; with the rows of level groups it is
 * the LB+LG traversal of Sec. 4.2.1 (Fig. 7b).  Y must hold pm blocks. */
void oracle_lb_mpk(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                   int32_t nunits, const int32_t *unit_ptr, int32_t pm, int32_t nrhs,
                   const double *x, double *Y)
{
    const int64_t blk = (int64_t)n * nrhs;
    for (int32_t d = 1; d <= nunits + pm - 1; d++) {
        int32_t p_start = (d - nunits + 1 > 1) ? d - nunits + 1 : 1;
        int32_t p_end = (d < pm) ? d : pm;
        for (int32_t p = p_start; p <= p_end; p++) {
            int32_t i = d - p;
            const double *in = (p == 1) ? x : Y + (int64_t)(p - 2) * blk;
            if (unit_ptr[i + 1] > unit_ptr[i])
                oracle_spmv_rows(rowptr, col, val, nrhs, in, Y + (int64_t)(p - 1) * blk,
                                 unit_ptr[i], unit_ptr[i + 1] - 1);
        }
    }
}

/* ------------------------------------------------------------------ Krylov consumers of the MPK
 * Sec. 1 and Sec. 8 name s-step Krylov methods as users of the MPK: their
 * Krylov basis of s powers comes from one MPK.  Two FP64 references for a
 * symmetric positive definite A, both stopping when ||r|| <= tol ||b||:
 *
 * Conjugate gradients (Hestenes and Stiefel, 1952): r = b - A x, p = r; per
 * step q = A p, alpha = (r.r)/(p.q), x += alpha p, r -= alpha q,
 * beta = (r.r)_new/(r.r)_old, p = r + beta p.  Returns the steps taken;
 * *relres = ||r|| / ||b|| of the recurred residual.
 */
static double dotv(int32_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

int32_t oracle_cg(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, const double *b,
                  double *x, double tol, int32_t max_iter, double *relres)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)n), *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    oracle_spmv_rows(rowptr, col, val, 1, x, q, 0, n - 1);
    for (int32_t i = 0; i < n; i++) { r[i] = b[i] - q[i]; p[i] = r[i]; }
    const double bn = sqrt(dotv(n, b, b));
    double rr = dotv(n, r, r);
    int32_t it = 0;
    while (it < max_iter && !(sqrt(rr) <= tol * bn)) {
        oracle_spmv_rows(rowptr, col, val, 1, p, q, 0, n - 1);
        const double alpha = rr / dotv(n, p, q);
        for (int32_t i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        const double rr2 = dotv(n, r, r);
        const double beta = rr2 / rr;
        for (int32_t i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
        rr = rr2;
        it++;
    }
    *relres = bn > 0.0 ? sqrt(rr) / bn : 0.0;
    free(r); free(p); free(q);
    return it;
}

/* s-step conjugate gradients with the monomial basis (the communication-
 * avoiding CG of Hoemmen's and Carson's work, restated): an outer iteration
 * builds V = [p, Ap/rho, .., A^s p/rho^s, r, Ar/rho, .., A^(s-1) r/rho^(s-1)]
 * with one MPK of [p r], its Gram matrix G = V^T V, and runs s CG steps on
 * coordinate vectors of length 2s+1: with B the matrix of A in the basis
 * (B[j+1][j] = rho inside each block), p' = e_0, r' = e_(s+1), x' = 0:
 *   w = B p', alpha = (r'^T G r') / (p'^T G w), x' += alpha p',
 *   r'' = r' - alpha w, beta = (r''^T G r'') / (r'^T G r'), p' = r'' + beta p',
 * then x += V x', r = V r', p = V p'.  ||r||^2 = r'^T G r' gives the stop
 * test after every inner step.  Returns the CG steps taken.
 */
int32_t oracle_sstep_cg(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val, const double *b,
                        double *x, int32_t s, double rho, double tol, int32_t max_steps, double *relres)
{
    const int32_t m = 2 * s + 1;
    double *r = (double *)malloc(sizeof(double) * (size_t)n), *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *V = (double *)malloc(sizeof(double) * (size_t)n * m);
    double *Y = (double *)malloc(sizeof(double) * (size_t)n * s);
    double *G = (double *)malloc(sizeof(double) * (size_t)m * m);
    double xc[64], rc[64], pc[64], w[64], r2[64], Gv[64];
    oracle_spmv_rows(rowptr, col, val, 1, x, r, 0, n - 1);
    for (int32_t i = 0; i < n; i++) { r[i] = b[i] - r[i]; p[i] = r[i]; }
    const double bn = sqrt(dotv(n, b, b));
    double rr = dotv(n, r, r);
    int32_t steps = 0;
    while (steps < max_steps && !(sqrt(rr) <= tol * bn)) {
        /* the basis: powers of p (0..s) and of r (0..s-1), scaled by rho^-k */
        oracle_mpk(n, rowptr, col, val, s, 1, p, Y);
        for (int32_t i = 0; i < n; i++) V[(size_t)i * m] = p[i];
        for (int32_t k = 1; k <= s; k++)
            for (int32_t i = 0; i < n; i++) V[(size_t)i * m + k] = Y[(size_t)(k - 1) * n + i] / pow(rho, k);
        oracle_mpk(n, rowptr, col, val, s, 1, r, Y);
        for (int32_t i = 0; i < n; i++) V[(size_t)i * m + s + 1] = r[i];
        for (int32_t k = 1; k < s; k++)
            for (int32_t i = 0; i < n; i++) V[(size_t)i * m + s + 1 + k] = Y[(size_t)(k - 1) * n + i] / pow(rho, k);
        for (int32_t a = 0; a < m; a++)
            for (int32_t c = 0; c < m; c++) {
                double t = 0.0;
                for (int32_t i = 0; i < n; i++) t += V[(size_t)i * m + a] * V[(size_t)i * m + c];
                G[a * m + c] = t;
            }
        for (int32_t j = 0; j < m; j++) { xc[j] = 0.0; pc[j] = 0.0; rc[j] = 0.0; }
        pc[0] = 1.0;
        rc[s + 1] = 1.0;
        for (int32_t j = 0; j < s && steps < max_steps && !(sqrt(rr) <= tol * bn); j++) {
            for (int32_t a = 0; a < m; a++) w[a] = 0.0;
            for (int32_t a = 0; a < s; a++) w[a + 1] += rho * pc[a];                 /* the p block */
            for (int32_t a = 0; a < s - 1; a++) w[s + 2 + a] += rho * pc[s + 1 + a];  /* the r block */
            for (int32_t a = 0; a < m; a++) { Gv[a] = 0.0; for (int32_t c = 0; c < m; c++) Gv[a] += G[a * m + c] * w[c]; }
            double pGw = 0.0, rGr = 0.0;
            for (int32_t a = 0; a < m; a++) pGw += pc[a] * Gv[a];
            for (int32_t a = 0; a < m; a++) { double t = 0.0; for (int32_t c = 0; c < m; c++) t += G[a * m + c] * rc[c]; rGr += rc[a] * t; }
            const double alpha = rGr / pGw;
            for (int32_t a = 0; a < m; a++) { xc[a] += alpha * pc[a]; r2[a] = rc[a] - alpha * w[a]; }
            double rGr2 = 0.0;
            for (int32_t a = 0; a < m; a++) { double t = 0.0; for (int32_t c = 0; c < m; c++) t += G[a * m + c] * r2[c]; rGr2 += r2[a] * t; }
            const double beta = rGr2 / rGr;
            for (int32_t a = 0; a < m; a++) { pc[a] = r2[a] + beta * pc[a]; rc[a] = r2[a]; }
            rr = rGr2 > 0.0 ? rGr2 : 0.0;
            steps++;
        }
        for (int32_t i = 0; i < n; i++) {
            double dx = 0.0, nr = 0.0, np = 0.0;
            for (int32_t a = 0; a < m; a++) {
                const double v = V[(size_t)i * m + a];
                dx += xc[a] * v; nr += rc[a] * v; np += pc[a] * v;
            }
            x[i] += dx; r[i] = nr; p[i] = np;
        }
    }
    *relres = bn > 0.0 ? sqrt(dotv(n, r, r)) / bn : 0.0;
    free(r); free(p); free(V); free(Y); free(G);
    return steps;
}

/* ------------------------------------------------------------------ Chebyshev
 * Gershgorin interval of A: [min_i (a_ii - sum_{j!=i} |a_ij|),
 * max_i (a_ii + sum_{j!=i} |a_ij|)].  Reading of the spectral scaling the
 * paper leaves unstated (Sec. 7): centre c = (hi+lo)/2, half-width r = (hi-lo)/2. */
void oracle_gershgorin(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                       double *lo, double *hi)
{
    double l = INFINITY, h = -INFINITY;
    for (int32_t i = 0; i < n; i++) {
        double d = 0.0, s = 0.0;
        for (int32_t e = rowptr[i]; e < rowptr[i + 1]; e++) {
            if (col[e] == i) d += val[e]; else s += fabs(val[e]);
        }
        if (d - s < l) l = d - s;
        if (d + s > h) h = d + s;
    }
    *lo = l; *hi = h;
}

/* Schroedinger propagator coefficients (hbar = 1): with H = c + r*Ahat,
 * exp(-i H dt) = exp(-i c dt) [ J_0(r dt) T_0(Ahat) + 2 sum_{k>=1} (-i)^k J_k(r dt) T_k(Ahat) ]
 * (Jacobi-Anger expansion; the Bessel-function coefficients of Sec. 7).
 * coef holds M+1 complex numbers, interleaved (re, im). */
void oracle_cheb_coeffs_schroedinger(int32_t M, double c, double r, double dt, double *coef)
{
    double ph_re = cos(c * dt), ph_im = -sin(c * dt);   /* exp(-i c dt) */
    for (int32_t k = 0; k <= M; k++) {
        double a = (k == 0 ? 1.0 : 2.0) * jn(k, r * dt);
        double mi_re, mi_im;                               /* (-i)^k */
        switch (k & 3) {
        case 0: mi_re = 1.0;  mi_im = 0.0;  break;
        case 1: mi_re = 0.0;  mi_im = -1.0; break;
        case 2: mi_re = -1.0; mi_im = 0.0;  break;
        default: mi_re = 0.0; mi_im = 1.0;  break;
        }
        double t_re = a * mi_re, t_im = a * mi_im;
        coef[2 * k]     = ph_re * t_re - ph_im * t_im;
        coef[2 * k + 1] = ph_re * t_im + ph_im * t_re;
    }
}

/* Chebyshev time propagation (Sec. 7, Eq. 7-9) for a real matrix A and a
 * complex vector x (interleaved re, im; row-major n x 2):
 *   Ahat = (A - c I) / r,  v_0 = x,  v_1 = Ahat v_0,
 *   v_{k+1} = 2 Ahat v_k - v_{k-1},  y = sum_{k=0}^{M} coef_k v_k,
 * with complex coef (interleaved).  All arithmetic in FP64. */
void oracle_cheb(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                 double c, double r, int32_t M, const double *coef, const double *x, double *y)
{
    const int64_t len = (int64_t)n * 2;
    double *vprev = (double *)malloc(sizeof(double) * (size_t)(len > 0 ? len : 1));
    double *vcur  = (double *)malloc(sizeof(double) * (size_t)(len > 0 ? len : 1));
    double *av    = (double *)malloc(sizeof(double) * (size_t)(len > 0 ? len : 1));
    memcpy(vprev, x, sizeof(double) * (size_t)len);
    for (int64_t i = 0; i < n; i++) {              /* y = coef_0 * v_0 */
        double vr = x[2 * i], vi = x[2 * i + 1];
        y[2 * i]     = coef[0] * vr - coef[1] * vi;
        y[2 * i + 1] = coef[0] * vi + coef[1] * vr;
    }
    for (int32_t k = 1; k <= M; k++) {
        const double *src = (k == 1) ? vprev : vcur;
        if (n > 0) oracle_spmv_rows(rowptr, col, val, 2, src, av, 0, n - 1);
        for (int64_t i = 0; i < len; i++) {
            double ah = (av[i] - c * src[i]) / r;  /* Ahat v */
            double vnew = (k == 1) ? ah : 2.0 * ah - vprev[i];
            if (k > 1) vprev[i] = vcur[i];
            vcur[i] = vnew;
        }
        const double cr = coef[2 * k], ci = coef[2 * k + 1];
        for (int64_t i = 0; i < n; i++) {
            double vr = vcur[2 * i], vi = vcur[2 * i + 1];
            y[2 * i]     += cr * vr - ci * vi;
            y[2 * i + 1] += cr * vi + ci * vr;
        }
    }
    free(vprev); free(vcur); free(av);
}

/* Heat-equation propagator coefficients (Sec. 7, the modified-Bessel case):
 * with A = c + r*Ahat and tau = a*dt,
 *   exp(-tau A) = exp(-tau c) [ I_0(tau r) T_0(Ahat) + 2 sum_{k>=1} (-1)^k I_k(tau r) T_k(Ahat) ],
 * the generating function exp(z cos t) = I_0(z) + 2 sum_k I_k(z) cos(k t) taken at
 * z = -tau r (I_k(-z) = (-1)^k I_k(z)).  The scaled values I_k(z) e^{-z} come from
 * the integral (1/pi) int_0^pi exp(z (cos t - 1)) cos(k t) dt, evaluated with the
 * trapezoid rule on nq panels (exponentially convergent for this periodic,
 * analytic integrand); exp(-tau c) I_k(z) = exp(-tau (c - r)) * I_k(z) e^{-z}.
 * coef holds M+1 real numbers. */
void oracle_cheb_coeffs_heat(int32_t M, double c, double r, double tau, double *coef)
{
    const double z = tau * r, pi = acos(-1.0);
    const int32_t nq = 8192 + 8 * M + (int32_t)(16.0 * sqrt(z + 1.0));
    const double scale = exp(-tau * (c - r));
    for (int32_t k = 0; k <= M; k++) {
        double s = 0.0;
        for (int32_t j = 0; j <= nq; j++) {
            const double t = pi * (double)j / (double)nq;
            const double f = exp(z * (cos(t) - 1.0)) * cos((double)k * t);
            s += (j == 0 || j == nq) ? 0.5 * f : f;
        }
        const double ive = s / (double)nq;
        coef[k] = (k == 0 ? 1.0 : 2.0) * ((k & 1) ? -1.0 : 1.0) * scale * ive;
    }
}

/* Chebyshev time propagation (Sec. 7, Eq. 7-9) for a real matrix A and a
 * real vector x: Ahat = (A - c I) / r, v_0 = x, v_1 = Ahat v_0,
 * v_{k+1} = 2 Ahat v_k - v_{k-1}, y = sum_{k=0}^{M} coef_k v_k (coef real).
 * All arithmetic in FP64. */
void oracle_cheb_real(int32_t n, const int32_t *rowptr, const int32_t *col, const double *val,
                      double c, double r, int32_t M, const double *coef, const double *x, double *y)
{
    const size_t len = (size_t)(n > 0 ? n : 1);
    double *vprev = (double *)malloc(sizeof(double) * len);
    double *vcur  = (double *)malloc(sizeof(double) * len);
    double *av    = (double *)malloc(sizeof(double) * len);
    memcpy(vprev, x, sizeof(double) * (size_t)n);
    for (int32_t i = 0; i < n; i++) y[i] = coef[0] * x[i];
    for (int32_t k = 1; k <= M; k++) {
        const double *src = (k == 1) ? vprev : vcur;
        if (n > 0) oracle_spmv_rows(rowptr, col, val, 1, src, av, 0, n - 1);
        for (int32_t i = 0; i < n; i++) {
            double ah = (av[i] - c * src[i]) / r;   /* Ahat v */
            double vnew = (k == 1) ? ah : 2.0 * ah - vprev[i];
            if (k > 1) vprev[i] = vcur[i];
            vcur[i] = vnew;
        }
        for (int32_t i = 0; i < n; i++) y[i] += coef[k] * vcur[i];
    }
    free(vprev); free(vcur); free(av);
}
