/*
 * uaamg_oracle.c -- plain, serial, FP64 CPU statement of unsmoothed-aggregation AMG
 * (Brannick, Chen, Hu, Zikatanov, "Parallel Unsmoothed Aggregation Algebraic Multigrid
 * Algorithms on GPUs").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is checked
 * against.  Only the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  The product library never links, loads or calls it, and it shares no code,
 * header, table or helper with the CUDA sources.
 *
 * Every routine is written for a reader checking it against the paper by eye: no blocking,
 * no fusion, no reordering beyond what the cited passage states.  Floating point is FP64
 * throughout, and the file is compiled with -ffp-contract=off so that x86 and Arm hosts
 * produce the same bits.
 *
 * Readings of the paper where it is silent or ambiguous (each is pinned by a test):
 *  - Priority (Eq. 3.2): rand() is replaced by a seeded bijective hash h_i in [0, 2^32), and
 *    v_i = d_i + ((i mod 12) + h_i / 2^32) / 12 is encoded exactly as the integer
 *    P_i = ((12 d_i + (i mod 12) + 1) << 32) | h_i.  Larger P = higher priority; the hash
 *    is a bijection, so priorities are unique and no tie-break is needed.
 *  - Coarse vertices per pass (Section 3.1, Algorithm 2): a maximal distance-2 independent
 *    set of the unprocessed vertices, where distance is measured in the whole graph of the
 *    current level (paths may pass through processed vertices).  It is computed as the
 *    greedy scan in descending priority.  The literal one-round variant of Algorithm 2
 *    (step 2b applied once per pass) is available as pass mode 1.
 *  - Aggregates (Algorithm 2 step 2c, Section 3.1): a root plus its unprocessed distance-1
 *    neighbours, taken in ascending index, at most t vertices in total (t = 0: no limit).
 *  - Coarse numbering (Section 5.1): the k-th root in ascending vertex index is coarse
 *    vertex k.
 *  - Levels are numbered 0 = finest.  Coarsening continues while n_l > coarse_size and the
 *    level count is below max_levels (Algorithm 1 setup loop).
 *  - Aggregating twice per level (Section 3.3, equivalent to skipping a level): the second
 *    stage aggregates the first stage's coarse matrix with priority salt index 2l+1 (the
 *    first stage uses 2l), and is skipped when that matrix is already <= coarse_size.
 *  - K-cycle (Section 4.3): two flexible-CG steps on each coarse level, preconditioned by
 *    the next level's cycle, with the coarsest level solved exactly by dense Cholesky.
 *    Optional safeguards the paper does not state (both off by default): one step only on
 *    levels reached by weak coarsening (kcycle_ratio), and stopping the hierarchy when a
 *    small level stops coarsening (min_coarsening).
 *  - Outer iteration (Section 1, Section 4.4): flexible CG with one stored direction,
 *    preconditioned by the K-cycle, stopped on the relative l2 residual of b - A x.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NOT_SPD 3
#define OR_ERR_NO_CONVERGENCE 4
#define OR_ERR_OOM 5
#define OR_ERR_UNSUPPORTED 9

#define OR_MAX_LEVELS 64
#define OR_MAX_COARSEST 4096

/* ------------------------------------------------------------------------------------ */
/* Priority vector, Eq. (3.2)                                                           */
/* ------------------------------------------------------------------------------------ */

/* MurmurHash3 32-bit finalizer (Appleby, 2011): xor-shift / odd-multiply steps, each of
 * which is invertible on 32-bit words, so the whole map is a bijection. */
uint32_t or_fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

/* Per-level salt added to the vertex index before hashing. */
uint32_t or_level_salt(uint64_t seed, int32_t level) {
    uint32_t s = (uint32_t)(seed ^ (seed >> 32));
    return s + 0x9E3779B9u * (uint32_t)level;
}

/* P_i for every vertex of a level.  d_i = number of stored off-diagonal entries of row i. */
void or_priorities(int32_t n, const int32_t* rowptr, const int32_t* col, uint64_t seed,
                   int32_t level, uint64_t* P) {
    uint32_t salt = or_level_salt(seed, level);
    for (int32_t i = 0; i < n; i++) {
        int64_t d = 0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++)
            if (col[k] != i) d++;
        uint64_t band = (uint64_t)(12 * d + (i % 12) + 1);
        P[i] = (band << 32) | (uint64_t)or_fmix32((uint32_t)i + salt);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Parallel aggregation algorithm, Algorithm 2, stated serially                          */
/* ------------------------------------------------------------------------------------ */

static const uint64_t* g_sort_keys; /* qsort has no context argument */
static int cmp_desc_priority(const void* a, const void* b) {
    uint64_t pa = g_sort_keys[*(const int32_t*)a], pb = g_sort_keys[*(const int32_t*)b];
    return (pa < pb) ? 1 : (pa > pb) ? -1 : 0;
}

/* Marks every vertex at graph distance <= 2 from i with `token`. */
static void mark_distance2(const int32_t* rowptr, const int32_t* col, int32_t i, int32_t token,
                           int32_t* mark) {
    mark[i] = token;
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
        int32_t u = col[k];
        mark[u] = token;
        for (int32_t q = rowptr[u]; q < rowptr[u + 1]; q++) mark[col[q]] = token;
    }
}

/* True iff P_i exceeds P_w for every unprocessed w != i within distance 2 of i
 * (Algorithm 2 step 2b). */
static int is_local_max(const int32_t* rowptr, const int32_t* col, const uint64_t* P,
                        const int32_t* root_of, int32_t i) {
    for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
        int32_t u = col[k];
        if (u != i && root_of[u] < 0 && P[u] > P[i]) return 0;
        for (int32_t q = rowptr[u]; q < rowptr[u + 1]; q++) {
            int32_t w = col[q];
            if (w != i && root_of[w] < 0 && P[w] > P[i]) return 0;
        }
    }
    return 1;
}

/*
 * Algorithm 2 as passes of (A) coarse-vertex selection and (B) aggregation, until every
 * vertex belongs to an aggregate.  t = 0: no size limit, t >= 2: at most t vertices per
 * aggregate.  mode 0: maximal set per pass (greedy in descending priority); mode 1: one
 * round of local maxima per pass.
 * Outputs root_of[i] (the root of i's aggregate) and pass_of[i] (the pass in which i was
 * aggregated).  Returns the number of passes, or -1 on a bad argument.
 */
int32_t or_paa(int32_t n, const int32_t* rowptr, const int32_t* col, const uint64_t* P,
               int32_t t, int32_t mode, int32_t* root_of, int32_t* pass_of) {
    if (n < 0 || t < 0 || t == 1 || (mode != 0 && mode != 1)) return -1;
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* roots = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < n; i++) {
        order[i] = i;
        mark[i] = -1;
        root_of[i] = -1;
        pass_of[i] = -1;
    }
    g_sort_keys = P;
    qsort(order, (size_t)n, sizeof(int32_t), cmp_desc_priority);

    int32_t remaining = n, pass = 0;
    while (remaining > 0) {
        /* (A) coarse vertices of this pass */
        int32_t nroots = 0;
        if (mode == 0) {
            for (int32_t q = 0; q < n; q++) {
                int32_t i = order[q];
                if (root_of[i] >= 0 || mark[i] == pass) continue;
                roots[nroots++] = i;
                mark_distance2(rowptr, col, i, pass, mark);
            }
        } else {
            for (int32_t i = 0; i < n; i++)
                if (root_of[i] < 0 && is_local_max(rowptr, col, P, root_of, i)) roots[nroots++] = i;
        }
        /* (B) each root takes itself and its unprocessed neighbours, ascending, up to t */
        for (int32_t r = 0; r < nroots; r++) {
            int32_t c = roots[r];
            root_of[c] = c;
            pass_of[c] = pass;
            int32_t taken = 1;
            for (int32_t k = rowptr[c]; k < rowptr[c + 1]; k++) {
                int32_t u = col[k];
                if (u == c || root_of[u] >= 0) continue;
                if (t > 0 && taken >= t) break;
                root_of[u] = c;
                pass_of[u] = pass;
                taken++;
            }
            remaining -= taken;
        }
        pass++;
    }
    free(order);
    free(mark);
    free(roots);
    return pass;
}

/* Coarse numbering, Section 5.1: roots in ascending index get 0, 1, 2, ...
 * agg[i] = coarse index of i's aggregate (the column of P holding row i).  Returns n_c. */
int32_t or_renumber(int32_t n, const int32_t* root_of, int32_t* agg) {
    int32_t* cid = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t nc = 0;
    for (int32_t i = 0; i < n; i++) cid[i] = (root_of[i] == i) ? nc++ : -1;
    for (int32_t i = 0; i < n; i++) agg[i] = cid[root_of[i]];
    free(cid);
    return nc;
}

/* ------------------------------------------------------------------------------------ */
/* Coarse operator, Eq. (2.4)                                                            */
/* ------------------------------------------------------------------------------------ */

static int cmp_int32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/*
 * (A_c)_IJ = sum over s in G_I, t in G_J of a_st.  The pattern is every pair (agg[s], agg[t])
 * of a stored entry (s, t) -- structural, nothing is dropped -- with columns sorted.  Each
 * sum starts at +0.0 and adds the entries in fine CSR order (ascending s, then stored
 * order).  cap = capacity of col_c / val_c.  Returns nnz_c, or -1 if cap is too small.
 */
int64_t or_coarse(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                  const int32_t* agg, int32_t nc, int32_t* rowptr_c, int32_t* col_c,
                  double* val_c, int64_t cap) {
    /* members of each aggregate in ascending fine index (transpose of P) */
    int32_t* mptr = (int32_t*)calloc((size_t)nc + 1, sizeof(int32_t));
    int32_t* mem = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
    for (int32_t i = 0; i < n; i++) mptr[agg[i] + 1]++;
    for (int32_t I = 0; I < nc; I++) mptr[I + 1] += mptr[I];
    for (int32_t I = 0; I < nc; I++) fill[I] = mptr[I];
    for (int32_t i = 0; i < n; i++) mem[fill[agg[i]]++] = i;

    double* acc = (double*)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
    int32_t* seen = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
    for (int32_t J = 0; J < nc; J++) seen[J] = -1;

    int64_t pos = 0;
    rowptr_c[0] = 0;
    for (int32_t I = 0; I < nc; I++) {
        int32_t cnt = 0;
        for (int32_t m = mptr[I]; m < mptr[I + 1]; m++) {
            int32_t s = mem[m];
            for (int32_t k = rowptr[s]; k < rowptr[s + 1]; k++) {
                int32_t J = agg[col[k]];
                if (seen[J] != I) {
                    seen[J] = I;
                    acc[J] = 0.0;
                    list[cnt++] = J;
                }
                acc[J] += val[k];
            }
        }
        qsort(list, (size_t)cnt, sizeof(int32_t), cmp_int32);
        if (pos + cnt > cap) {
            pos = -1;
            break;
        }
        for (int32_t q = 0; q < cnt; q++) {
            col_c[pos] = list[q];
            val_c[pos] = acc[list[q]];
            pos++;
        }
        rowptr_c[I + 1] = (int32_t)pos;
    }
    free(mptr);
    free(mem);
    free(fill);
    free(acc);
    free(seen);
    free(list);
    return pos;
}

/* ------------------------------------------------------------------------------------ */
/* l1-Jacobi smoother, Section 4.1                                                       */
/* ------------------------------------------------------------------------------------ */

/* Damped Jacobi (Section 4.1): Minv_i = omega / a_ii. */
void or_minv_damped(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                    double omega, double* minv) {
    for (int32_t i = 0; i < n; i++) {
        double diag = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++)
            if (col[k] == i) diag = val[k];
        minv[i] = omega / diag;
    }
}

/* Minv_i = 1 / (a_ii + sum_{j != i} |a_ij|), the row sum taken in stored order. */
void or_minv(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
             double* minv) {
    for (int32_t i = 0; i < n; i++) {
        double diag = 0.0, off = 0.0;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
            if (col[k] == i) diag = val[k];
            else off += fabs(val[k]);
        }
        minv[i] = 1.0 / (diag + off);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Coarsest-level exact solve, Algorithm 1 ("solve exactly"): dense Cholesky              */
/* ------------------------------------------------------------------------------------ */

/* In-place Cholesky A = L L^T of a row-major m x m SPD matrix; the lower triangle of A is
 * overwritten by L.  Returns 0, or -(j+1) when pivot j is not positive. */
int32_t or_cholesky(int32_t m, double* A) {
    for (int32_t j = 0; j < m; j++) {
        double s = A[(size_t)j * m + j];
        for (int32_t k = 0; k < j; k++) s -= A[(size_t)j * m + k] * A[(size_t)j * m + k];
        if (!(s > 0.0)) return -(j + 1);
        double ljj = sqrt(s);
        A[(size_t)j * m + j] = ljj;
        for (int32_t i = j + 1; i < m; i++) {
            double v = A[(size_t)i * m + j];
            for (int32_t k = 0; k < j; k++) v -= A[(size_t)i * m + k] * A[(size_t)j * m + k];
            A[(size_t)i * m + j] = v / ljj;
        }
    }
    return 0;
}

/* Solves L L^T x = b with the factor from or_cholesky. */
void or_cholesky_solve(int32_t m, const double* L, const double* b, double* x) {
    for (int32_t i = 0; i < m; i++) {
        double v = b[i];
        for (int32_t k = 0; k < i; k++) v -= L[(size_t)i * m + k] * x[k];
        x[i] = v / L[(size_t)i * m + i];
    }
    for (int32_t i = m - 1; i >= 0; i--) {
        double v = x[i];
        for (int32_t k = i + 1; k < m; k++) v -= L[(size_t)k * m + i] * x[k];
        x[i] = v / L[(size_t)i * m + i];
    }
}

/* ------------------------------------------------------------------------------------ */
/* Hierarchy, Algorithm 1 setup phase                                                    */
/* ------------------------------------------------------------------------------------ */

typedef struct or_params {
    int32_t coarse_size;  /* coarsen while n_l > coarse_size */
    int32_t max_levels;   /* at most this many levels, finest included */
    int32_t max_agg_size; /* t: 0 = unbounded, else >= 2 */
    int32_t pass_mode;    /* 0 maximal per pass, 1 one round per pass */
    uint64_t seed;        /* hash seed of the priority vector */
    int32_t pre, post;    /* l1-Jacobi sweeps before / after the coarse correction */
    int32_t kcycle_inner; /* 1 or 2 flexible-CG steps per coarse level */
    double kcycle_tau;    /* > 0: skip the second step when |rho~| <= tau |rho| */
    int32_t max_iter;     /* outer iterations */
    int32_t agg_repeat;   /* 1: one aggregation per level; 2: aggregate twice (Section 3.3) */
    double kcycle_ratio;  /* > 0: level m takes its second step only if n_{m-1}/n_m >= this */
    double min_coarsening; /* > 0: a level with n <= 1024 that would shrink by less than this
                              factor becomes the coarsest */
    double jacobi_omega;  /* 0: l1-Jacobi; > 0: damped Jacobi x += omega D^{-1} (b - A x) */
} or_params;

typedef struct or_level {
    int32_t n;
    int64_t nnz;
    int32_t *rowptr, *col;
    double *val, *minv;
    int32_t* agg;     /* fine -> coarse map to the next level (NULL on the coarsest) */
    int32_t* pass_of; /* pass in which each vertex was aggregated */
    int32_t nc, passes;
} or_level;

typedef struct or_hier {
    or_params p;
    int32_t nlev;
    or_level lev[OR_MAX_LEVELS];
    double* chol; /* dense Cholesky factor of the coarsest matrix */
} or_hier;

void or_free(void* hv);

void* or_setup(int32_t n, const int32_t* rowptr, const int32_t* col, const double* val,
               const or_params* p, int32_t* status) {
    *status = OR_ERR_ARG;
    if (n < 1 || p->coarse_size < 1 || p->max_levels < 1 || p->max_levels > OR_MAX_LEVELS ||
        p->max_agg_size < 0 || p->max_agg_size == 1 || p->pre < 0 || p->post < 0 ||
        p->kcycle_inner < 1 || p->kcycle_inner > 2 || p->max_iter < 0 ||
        p->agg_repeat < 1 || p->agg_repeat > 2 || p->kcycle_ratio < 0 || p->min_coarsening < 0 ||
        p->jacobi_omega < 0)
        return NULL;
    or_hier* h = (or_hier*)calloc(1, sizeof(or_hier));
    h->p = *p;
    or_level* L0 = &h->lev[0];
    L0->n = n;
    L0->nnz = rowptr[n];
    L0->rowptr = (int32_t*)malloc(sizeof(int32_t) * ((size_t)n + 1));
    L0->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(L0->nnz > 0 ? L0->nnz : 1));
    L0->val = (double*)malloc(sizeof(double) * (size_t)(L0->nnz > 0 ? L0->nnz : 1));
    memcpy(L0->rowptr, rowptr, sizeof(int32_t) * ((size_t)n + 1));
    memcpy(L0->col, col, sizeof(int32_t) * (size_t)L0->nnz);
    memcpy(L0->val, val, sizeof(double) * (size_t)L0->nnz);

    int32_t l = 0;
    while (h->lev[l].n > p->coarse_size && l + 1 < p->max_levels) {
        or_level* F = &h->lev[l];
        /* stage 1: aggregate the level's graph (priority salt index l, or 2l when twice) */
        const int32_t stage_salt = (p->agg_repeat == 2) ? 2 * l : l;
        uint64_t* P = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)F->n);
        int32_t* root_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)F->n);
        F->pass_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)F->n);
        F->agg = (int32_t*)malloc(sizeof(int32_t) * (size_t)F->n);
        or_priorities(F->n, F->rowptr, F->col, p->seed, stage_salt, P);
        F->passes = or_paa(F->n, F->rowptr, F->col, P, p->max_agg_size, p->pass_mode, root_of,
                           F->pass_of);
        F->nc = or_renumber(F->n, root_of, F->agg);
        free(P);
        free(root_of);
        if (F->nc == F->n) { /* no coarsening possible: this level is the coarsest */
            free(F->agg);
            F->agg = NULL;
            F->nc = 0;
            break;
        }
        or_level* C = &h->lev[l + 1];
        C->n = F->nc;
        C->rowptr = (int32_t*)malloc(sizeof(int32_t) * ((size_t)C->n + 1));
        C->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(F->nnz > 0 ? F->nnz : 1));
        C->val = (double*)malloc(sizeof(double) * (size_t)(F->nnz > 0 ? F->nnz : 1));
        C->nnz = or_coarse(F->n, F->rowptr, F->col, F->val, F->agg, F->nc, C->rowptr, C->col,
                           C->val, F->nnz);
        /* stage 2 (Section 3.3, aggregation applied twice = one level skipped): aggregate the
         * intermediate matrix C again; the level's aggregates are the unions, agg = agg2[agg1],
         * and the next matrix is Eq. (2.4) applied to C with agg2. */
        if (p->agg_repeat == 2 && C->n > p->coarse_size) {
            uint64_t* P2 = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)C->n);
            int32_t* root2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)C->n);
            int32_t* pass2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)C->n);
            int32_t* agg2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)C->n);
            or_priorities(C->n, C->rowptr, C->col, p->seed, 2 * l + 1, P2);
            or_paa(C->n, C->rowptr, C->col, P2, p->max_agg_size, p->pass_mode, root2, pass2);
            int32_t nc2 = or_renumber(C->n, root2, agg2);
            if (nc2 < C->n) {
                int32_t* rp2 = (int32_t*)malloc(sizeof(int32_t) * ((size_t)nc2 + 1));
                int32_t* col2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(C->nnz > 0 ? C->nnz : 1));
                double* val2 = (double*)malloc(sizeof(double) * (size_t)(C->nnz > 0 ? C->nnz : 1));
                int64_t z2 = or_coarse(C->n, C->rowptr, C->col, C->val, agg2, nc2, rp2, col2,
                                       val2, C->nnz);
                for (int32_t i = 0; i < F->n; i++) F->agg[i] = agg2[F->agg[i]];
                F->nc = nc2;
                free(C->rowptr);
                free(C->col);
                free(C->val);
                C->n = nc2;
                C->nnz = z2;
                C->rowptr = rp2;
                C->col = col2;
                C->val = val2;
            }
            free(P2);
            free(root2);
            free(pass2);
            free(agg2);
        }
        /* stagnating coarsening: keep this level as the coarsest when it is small enough */
        if (p->min_coarsening > 0.0 && F->n <= 1024 &&
            (double)F->n < p->min_coarsening * (double)F->nc) {
            free(C->rowptr);
            free(C->col);
            free(C->val);
            C->rowptr = NULL;
            C->col = NULL;
            C->val = NULL;
            C->n = 0;
            C->nnz = 0;
            free(F->agg);
            F->agg = NULL;
            F->nc = 0;
            break;
        }
        l++;
    }
    h->nlev = l + 1;
    for (int32_t q = 0; q < h->nlev; q++) {
        or_level* Lq = &h->lev[q];
        Lq->minv = (double*)malloc(sizeof(double) * (size_t)Lq->n);
        if (p->jacobi_omega > 0.0)
            or_minv_damped(Lq->n, Lq->rowptr, Lq->col, Lq->val, p->jacobi_omega, Lq->minv);
        else
            or_minv(Lq->n, Lq->rowptr, Lq->col, Lq->val, Lq->minv);
    }
    or_level* Lc = &h->lev[h->nlev - 1];
    if (Lc->n > OR_MAX_COARSEST) {
        *status = OR_ERR_UNSUPPORTED;
        or_free(h);
        return NULL;
    }
    h->chol = (double*)calloc((size_t)Lc->n * Lc->n, sizeof(double));
    for (int32_t i = 0; i < Lc->n; i++)
        for (int32_t k = Lc->rowptr[i]; k < Lc->rowptr[i + 1]; k++)
            h->chol[(size_t)i * Lc->n + Lc->col[k]] = Lc->val[k];
    if (or_cholesky(Lc->n, h->chol) != 0) {
        *status = OR_ERR_NOT_SPD;
        or_free(h);
        return NULL;
    }
    *status = OR_OK;
    return h;
}

void or_free(void* hv) {
    or_hier* h = (or_hier*)hv;
    if (!h) return;
    for (int32_t q = 0; q < OR_MAX_LEVELS; q++) {
        or_level* L = &h->lev[q];
        free(L->rowptr);
        free(L->col);
        free(L->val);
        free(L->minv);
        free(L->agg);
        free(L->pass_of);
    }
    free(h->chol);
    free(h);
}

int32_t or_num_levels(void* hv) { return ((or_hier*)hv)->nlev; }
int32_t or_level_n(void* hv, int32_t l) { return ((or_hier*)hv)->lev[l].n; }
int64_t or_level_nnz(void* hv, int32_t l) { return ((or_hier*)hv)->lev[l].nnz; }
int32_t or_level_passes(void* hv, int32_t l) { return ((or_hier*)hv)->lev[l].passes; }

void or_level_csr(void* hv, int32_t l, int32_t* rowptr, int32_t* col, double* val) {
    or_level* L = &((or_hier*)hv)->lev[l];
    memcpy(rowptr, L->rowptr, sizeof(int32_t) * ((size_t)L->n + 1));
    memcpy(col, L->col, sizeof(int32_t) * (size_t)L->nnz);
    memcpy(val, L->val, sizeof(double) * (size_t)L->nnz);
}
void or_level_agg(void* hv, int32_t l, int32_t* agg) {
    or_level* L = &((or_hier*)hv)->lev[l];
    memcpy(agg, L->agg, sizeof(int32_t) * (size_t)L->n);
}
void or_level_pass_of(void* hv, int32_t l, int32_t* pass_of) {
    or_level* L = &((or_hier*)hv)->lev[l];
    memcpy(pass_of, L->pass_of, sizeof(int32_t) * (size_t)L->n);
}
void or_level_minv(void* hv, int32_t l, double* minv) {
    or_level* L = &((or_hier*)hv)->lev[l];
    memcpy(minv, L->minv, sizeof(double) * (size_t)L->n);
}

/* ------------------------------------------------------------------------------------ */
/* Solve phase: Algorithm 1 solve, K-cycle (Section 4.3), outer flexible CG               */
/* ------------------------------------------------------------------------------------ */

static void spmv(const or_level* L, const double* x, double* y) {
    for (int32_t i = 0; i < L->n; i++) {
        double s = 0.0;
        for (int32_t k = L->rowptr[i]; k < L->rowptr[i + 1]; k++) s += L->val[k] * x[L->col[k]];
        y[i] = s;
    }
}

static double dot(int32_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int32_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

static double* vec(int32_t n) { return (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

static void apply_K(const or_hier* h, int32_t m, const double* rho, double* e);

/* One l1-Jacobi sweep x <- x + Minv (r - A x). */
static void smooth(const or_level* L, const double* r, double* x, double* tmp) {
    spmv(L, x, tmp);
    for (int32_t i = 0; i < L->n; i++) x[i] = x[i] + L->minv[i] * (r[i] - tmp[i]);
}

/* x = B_l(r): the multigrid preconditioner at level l (Algorithm 1 solve phase), started
 * from x = 0, with the coarse problem handed to the K-cycle of level l+1. */
void or_apply_B(void* hv, int32_t l, const double* r, double* x) {
    const or_hier* h = (const or_hier*)hv;
    const or_level* L = &h->lev[l];
    int32_t n = L->n;
    if (l == h->nlev - 1) {
        or_cholesky_solve(n, h->chol, r, x);
        return;
    }
    double* tmp = vec(n);
    /* pre-smoothing from x = 0: the first sweep is x = Minv r */
    for (int32_t i = 0; i < n; i++) x[i] = 0.0;
    for (int32_t s = 0; s < h->p.pre; s++) smooth(L, r, x, tmp);
    /* restriction of the residual: r_c = P^T (r - A x) */
    const or_level* C = &h->lev[l + 1];
    double* rc = vec(C->n);
    double* ec = vec(C->n);
    spmv(L, x, tmp);
    for (int32_t i = 0; i < n; i++) rc[L->agg[i]] += r[i] - tmp[i];
    /* coarse-grid correction by the K-cycle of the next level */
    apply_K(h, l + 1, rc, ec);
    /* prolongation: (P e)_i = e_{agg[i]} */
    for (int32_t i = 0; i < n; i++) x[i] += ec[L->agg[i]];
    /* post-smoothing */
    for (int32_t s = 0; s < h->p.post; s++) smooth(L, r, x, tmp);
    free(tmp);
    free(rc);
    free(ec);
}

/* e = K_m(rho): approximate solve of A_m e = rho by at most two flexible-CG steps
 * preconditioned by B_m; exact on the coarsest level. */
static void apply_K(const or_hier* h, int32_t m, const double* rho, double* e) {
    const or_level* L = &h->lev[m];
    int32_t n = L->n;
    if (m == h->nlev - 1) {
        or_cholesky_solve(n, h->chol, rho, e);
        return;
    }
    double *c1 = vec(n), *v1 = vec(n), *rt = vec(n), *c2 = vec(n), *v2 = vec(n);
    or_apply_B((void*)h, m, rho, c1);
    spmv(L, c1, v1);
    double rho1 = dot(n, c1, v1), alpha1 = dot(n, c1, rho);
    if (!(rho1 > 0.0)) { /* rho = 0 or a breakdown: no correction */
        for (int32_t i = 0; i < n; i++) e[i] = 0.0;
        goto done;
    }
    double a1 = alpha1 / rho1;
    for (int32_t i = 0; i < n; i++) rt[i] = rho[i] - a1 * v1[i];
    int second = (h->p.kcycle_inner == 2);
    if (second && h->p.kcycle_ratio > 0.0 &&
        (double)h->lev[m - 1].n < h->p.kcycle_ratio * (double)L->n)
        second = 0; /* weak coarsening into level m: one step */
    if (second && h->p.kcycle_tau > 0.0) {
        double nr = sqrt(dot(n, rt, rt)), n0 = sqrt(dot(n, rho, rho));
        if (nr <= h->p.kcycle_tau * n0) second = 0;
    }
    if (second) {
        or_apply_B((void*)h, m, rt, c2);
        spmv(L, c2, v2);
        double gamma = dot(n, c2, v1), beta = dot(n, c2, v2), alpha2 = dot(n, c2, rt);
        double rho2 = beta - gamma * gamma / rho1;
        if (rho2 > 0.0) {
            double w1 = a1 - gamma * alpha2 / (rho1 * rho2), w2 = alpha2 / rho2;
            for (int32_t i = 0; i < n; i++) e[i] = w1 * c1[i] + w2 * c2[i];
            goto done;
        }
    }
    for (int32_t i = 0; i < n; i++) e[i] = a1 * c1[i];
done:
    free(c1);
    free(v1);
    free(rt);
    free(c2);
    free(v2);
}

void or_apply_K(void* hv, int32_t m, const double* rho, double* e) {
    apply_K((const or_hier*)hv, m, rho, e);
}

/*
 * Flexible CG preconditioned by B_0 (the "nonlinear preconditioned CG" of Sections 1 and
 * 4.4): p_k = z_k - ((z_k, q_{k-1}) / (p_{k-1}, q_{k-1})) p_{k-1}, q_k = A p_k,
 * alpha = (p_k, r_k) / (p_k, q_k).  Stops when |r| <= tol |b| for the recurrence residual
 * and then for the recomputed b - A x.  x holds the initial guess when use_guess != 0.
 * hist (length max_iter + 1, may be NULL) receives |r_k| / |b|.  Returns OR_OK or
 * OR_ERR_NO_CONVERGENCE (x = last iterate in both cases).
 */
int32_t or_solve(void* hv, const double* b, double* x, double tol, int32_t use_guess,
                 int32_t* iters, double* relres, double* hist) {
    const or_hier* h = (const or_hier*)hv;
    const or_level* L = &h->lev[0];
    int32_t n = L->n;
    double *r = vec(n), *z = vec(n), *p = vec(n), *q = vec(n), *ax = vec(n);
    if (!use_guess)
        for (int32_t i = 0; i < n; i++) x[i] = 0.0;
    double bn = sqrt(dot(n, b, b));
    spmv(L, x, ax);
    for (int32_t i = 0; i < n; i++) r[i] = b[i] - ax[i];
    double rn = sqrt(dot(n, r, r));
    int32_t status = OR_ERR_NO_CONVERGENCE, k = 0;
    double pq_prev = 0.0;
    if (bn == 0.0) {
        for (int32_t i = 0; i < n; i++) x[i] = 0.0;
        rn = 0.0;
        bn = 1.0;
    }
    if (hist) hist[0] = rn / bn;
    if (rn <= tol * bn) status = OR_OK;
    while (status != OR_OK && k < h->p.max_iter) {
        or_apply_B(hv, 0, r, z);
        if (k == 0) {
            for (int32_t i = 0; i < n; i++) p[i] = z[i];
        } else {
            double beta = dot(n, z, q) / pq_prev;
            for (int32_t i = 0; i < n; i++) p[i] = z[i] - beta * p[i];
        }
        spmv(L, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) break; /* loss of positive definiteness: stop with the last iterate */
        double alpha = dot(n, p, r) / pq;
        for (int32_t i = 0; i < n; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        pq_prev = pq;
        k++;
        rn = sqrt(dot(n, r, r));
        if (rn <= tol * bn) { /* confirm with the true residual */
            spmv(L, x, ax);
            for (int32_t i = 0; i < n; i++) r[i] = b[i] - ax[i];
            rn = sqrt(dot(n, r, r));
            if (rn <= tol * bn) status = OR_OK;
        }
        if (hist) hist[k] = rn / bn;
    }
    *iters = k;
    *relres = rn / bn;
    free(r);
    free(z);
    free(p);
    free(q);
    free(ax);
    return status;
}
