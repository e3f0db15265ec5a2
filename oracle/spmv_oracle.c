/*
 * CPU oracle for the row-partitioned sparse matrix-vector product of
 * "Machine Learning for CUDA+MPI Design Rules" (Pearson, Javeed, Devine),
 * Sec. III-A and Fig. 3.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or helper with the CUDA
 * path.  Plain sequential C, FP64 throughout, written for a reader to check
 * against the paper by eye: no blocking, no fusion, no reordering.
 *
 * What is computed (Sec. III-A):
 *   - y = A x for a CSR matrix, rows in order, entries of a row in order.
 *   - The partition of Fig. 3b: P ranks own contiguous, even row blocks
 *     r_p = floor(p n / P) .. r_{p+1}.  Rank p splits its rows into A_L
 *     (columns inside its own range, rebased so that x_L = x[r_p..]) and
 *     A_R (the remaining columns).  A = A_L + A_R.
 *   - x_R: the remote x entries rank p needs are the sorted distinct remote
 *     columns H_p ("A is static, so the entries that make up x_R are fixed").
 *     A_R's columns are renumbered to positions in H_p.
 *   - Pack (vertex 2 of Fig. 3c): each rank copies the subset of x_L every
 *     other rank needs into a send buffer.  The buffer is laid out
 *     destination-major, then source rank, then ascending column, so the
 *     part bound for rank p is exactly x[H_p] and the exchange is one copy.
 *   - y = A_L x_L + A_R x_R, the remote product formed once x_R is assembled.
 *
 * Index types: column indices are int32 (n < 2^31); row pointers int64.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

/* ------------------------------------------------------------------ */
/* Plain CSR product: the definition y_i = sum_j a_ij x_j.             */
/* ------------------------------------------------------------------ */
int orc_csr_spmv(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                 const double *vals, const double *x, double *y)
{
    if (n < 0) return ORC_EINVAL;
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
            s += vals[k] * x[col_idx[k]];
        y[i] = s;
    }
    return ORC_OK;
}

/* The same definition with the rows shared among `threads` OpenMP threads
 * (0: the runtime's default; built without OpenMP: one thread).  Each row
 * is summed exactly as above, so y is bit-identical to orc_csr_spmv.  Used
 * only to time the oracle on every host core. */
int orc_csr_spmv_rows_parallel(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                               const double *vals, const double *x, double *y, int threads)
{
    if (n < 0) return ORC_EINVAL;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(static)
#else
    (void)threads;
#endif
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
            s += vals[k] * x[col_idx[k]];
        y[i] = s;
    }
    return ORC_OK;
}

/* Threads orc_csr_spmv_rows_parallel runs with by default. */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Per-row magnitude sum_j |a_ij x_j|: the scale of the dot-product rounding
 * error bound used by the parity tolerance. */
int orc_csr_absdot(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                   const double *vals, const double *x, double *out)
{
    if (n < 0) return ORC_EINVAL;
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
            s += fabs(vals[k] * x[col_idx[k]]);
        out[i] = s;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* The partition plan of Fig. 3b.                                       */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t rows;        /* r_{p+1} - r_p */
    int64_t *l_ptr;      /* rows+1, local CSR row pointer from 0 */
    int32_t *l_col;      /* rebased columns, 0 <= c < rows */
    double *l_val;
    int64_t l_nnz;
    int64_t *r_ptr;      /* rows+1, remote CSR row pointer from 0 */
    int32_t *r_col;      /* positions in halo[] */
    double *r_val;
    int64_t r_nnz;
    int32_t *halo;       /* H_p: sorted distinct global remote columns */
    int64_t n_halo;
} orc_rank;

typedef struct {
    int64_t n;
    int P;
    int64_t *bounds;     /* P+1 row bounds r_p */
    orc_rank *rk;
    int64_t n_send;      /* total send-buffer length */
    int32_t *send_idx;   /* global x index of every send-buffer slot */
    int64_t *halo_off;   /* P+1: start of destination p's part */
    int64_t *seg_off;    /* P*P+1: start of segment (dst p, src q) at p*P+q */
    double *sendbuf;     /* packed values */
    double *recvbuf;     /* received values (x_R of every rank, concatenated) */
    double *yr;          /* scratch for the remote product of one rank */
} orc_plan;

static int cmp_i32(const void *a, const void *b)
{
    int32_t u = *(const int32_t *)a, v = *(const int32_t *)b;
    return (u > v) - (u < v);
}

/* Rank that owns global index c: the p with r_p <= c < r_{p+1}. */
static int owner_of(const orc_plan *pl, int64_t c)
{
    for (int p = 0; p < pl->P; p++)
        if (pl->bounds[p] <= c && c < pl->bounds[p + 1]) return p;
    return -1;
}

/* Position of c in the sorted distinct list h[0..m), or -1. */
static int64_t find_sorted(const int32_t *h, int64_t m, int32_t c)
{
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (h[mid] < c) lo = mid + 1; else hi = mid;
    }
    return (lo < m && h[lo] == c) ? lo : -1;
}

void orc_plan_destroy(orc_plan *pl)
{
    if (!pl) return;
    if (pl->rk) {
        for (int p = 0; p < pl->P; p++) {
            orc_rank *r = &pl->rk[p];
            free(r->l_ptr); free(r->l_col); free(r->l_val);
            free(r->r_ptr); free(r->r_col); free(r->r_val); free(r->halo);
        }
    }
    free(pl->rk); free(pl->bounds); free(pl->send_idx); free(pl->halo_off);
    free(pl->seg_off); free(pl->sendbuf); free(pl->recvbuf); free(pl->yr);
    free(pl);
}

static void *xcalloc(size_t count, size_t size)
{
    /* never a zero-byte request, so a NULL return always means no memory */
    return calloc(count ? count : 1, size ? size : 1);
}

int orc_plan_create(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                    const double *vals, int P, orc_plan **out)
{
    *out = NULL;
    if (n < 0 || P < 1) return ORC_EINVAL;
    for (int64_t i = 0; i < n; i++) {
        if (row_ptr[i + 1] < row_ptr[i]) return ORC_EINVAL;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++)
            if (col_idx[k] < 0 || col_idx[k] >= n) return ORC_EINVAL;
    }
    orc_plan *pl = (orc_plan *)xcalloc(1, sizeof(orc_plan));
    if (!pl) return ORC_ENOMEM;
    pl->n = n;
    pl->P = P;
    pl->bounds = (int64_t *)xcalloc((size_t)P + 1, sizeof(int64_t));
    pl->rk = (orc_rank *)xcalloc((size_t)P, sizeof(orc_rank));
    if (!pl->bounds || !pl->rk) { orc_plan_destroy(pl); return ORC_ENOMEM; }
    /* contiguous, even row blocks: r_p = floor(p n / P) */
    for (int p = 0; p <= P; p++) pl->bounds[p] = (int64_t)(((__int128)p * n) / P);

    for (int p = 0; p < P; p++) {
        orc_rank *r = &pl->rk[p];
        int64_t rb = pl->bounds[p], re = pl->bounds[p + 1];
        r->rows = re - rb;
        int64_t nnz_all = row_ptr[re] - row_ptr[rb];
        r->l_ptr = (int64_t *)xcalloc((size_t)r->rows + 1, sizeof(int64_t));
        r->r_ptr = (int64_t *)xcalloc((size_t)r->rows + 1, sizeof(int64_t));
        r->l_col = (int32_t *)xcalloc((size_t)nnz_all, sizeof(int32_t));
        r->l_val = (double *)xcalloc((size_t)nnz_all, sizeof(double));
        r->r_col = (int32_t *)xcalloc((size_t)nnz_all, sizeof(int32_t));
        r->r_val = (double *)xcalloc((size_t)nnz_all, sizeof(double));
        r->halo = (int32_t *)xcalloc((size_t)nnz_all, sizeof(int32_t));
        if (!r->l_ptr || !r->r_ptr || !r->l_col || !r->l_val || !r->r_col ||
            !r->r_val || !r->halo) { orc_plan_destroy(pl); return ORC_ENOMEM; }

        /* split every row: own range -> A_L (rebased), otherwise -> A_R */
        int64_t nl = 0, nr = 0;
        for (int64_t i = rb; i < re; i++) {
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
                int32_t c = col_idx[k];
                if (c >= rb && c < re) {
                    r->l_col[nl] = (int32_t)(c - rb);
                    r->l_val[nl] = vals[k];
                    nl++;
                } else {
                    r->r_col[nr] = c;  /* global for now */
                    r->r_val[nr] = vals[k];
                    nr++;
                }
            }
            r->l_ptr[i - rb + 1] = nl;
            r->r_ptr[i - rb + 1] = nr;
        }
        r->l_nnz = nl;
        r->r_nnz = nr;

        /* H_p: the distinct remote columns, ascending */
        memcpy(r->halo, r->r_col, (size_t)nr * sizeof(int32_t));
        qsort(r->halo, (size_t)nr, sizeof(int32_t), cmp_i32);
        int64_t m = 0;
        for (int64_t k = 0; k < nr; k++)
            if (m == 0 || r->halo[m - 1] != r->halo[k]) r->halo[m++] = r->halo[k];
        r->n_halo = m;

        /* column-compress A_R: global column -> position in H_p */
        for (int64_t k = 0; k < nr; k++) {
            int64_t pos = find_sorted(r->halo, m, r->r_col[k]);
            r->r_col[k] = (int32_t)pos;
        }
    }

    /* send lists, destination-major, then source rank, then ascending column */
    pl->halo_off = (int64_t *)xcalloc((size_t)P + 1, sizeof(int64_t));
    pl->seg_off = (int64_t *)xcalloc((size_t)P * P + 1, sizeof(int64_t));
    if (!pl->halo_off || !pl->seg_off) { orc_plan_destroy(pl); return ORC_ENOMEM; }
    int64_t total = 0;
    for (int p = 0; p < P; p++) total += pl->rk[p].n_halo;
    pl->n_send = total;
    pl->send_idx = (int32_t *)xcalloc((size_t)total, sizeof(int32_t));
    pl->sendbuf = (double *)xcalloc((size_t)total, sizeof(double));
    pl->recvbuf = (double *)xcalloc((size_t)total, sizeof(double));
    int64_t maxrows = 1;
    for (int p = 0; p < P; p++) if (pl->rk[p].rows > maxrows) maxrows = pl->rk[p].rows;
    pl->yr = (double *)xcalloc((size_t)maxrows, sizeof(double));
    if (!pl->send_idx || !pl->sendbuf || !pl->recvbuf || !pl->yr) {
        orc_plan_destroy(pl); return ORC_ENOMEM;
    }
    int64_t k = 0;
    for (int p = 0; p < P; p++) {
        pl->halo_off[p] = k;
        const orc_rank *r = &pl->rk[p];
        for (int q = 0; q < P; q++) {
            pl->seg_off[(int64_t)p * P + q] = k;
            for (int64_t j = 0; j < r->n_halo; j++)
                if (owner_of(pl, r->halo[j]) == q) pl->send_idx[k++] = r->halo[j];
        }
    }
    pl->halo_off[P] = k;
    pl->seg_off[(int64_t)P * P] = k;
    *out = pl;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* The four operations of one rank (Fig. 3c), run on the CPU.          */
/* ------------------------------------------------------------------ */

/* Pack for source rank q (q = -1: every rank): sendbuf[k] = x[send_idx[k]]
 * for every slot k that q owns. */
int orc_pack(orc_plan *pl, int q, const double *x)
{
    if (q < -1 || q >= pl->P) return ORC_EINVAL;
    for (int p = 0; p < pl->P; p++)
        for (int s = 0; s < pl->P; s++) {
            if (q >= 0 && s != q) continue;
            for (int64_t k = pl->seg_off[(int64_t)p * pl->P + s];
                 k < pl->seg_off[(int64_t)p * pl->P + s + 1]; k++)
                pl->sendbuf[k] = x[pl->send_idx[k]];
        }
    return ORC_OK;
}

/* Exchange into destination p (p = -1: every rank): the part of the send
 * buffer bound for p lands in p's receive buffer. */
int orc_copy(orc_plan *pl, int p)
{
    if (p < -1 || p >= pl->P) return ORC_EINVAL;
    for (int d = 0; d < pl->P; d++) {
        if (p >= 0 && d != p) continue;
        for (int64_t k = pl->halo_off[d]; k < pl->halo_off[d + 1]; k++)
            pl->recvbuf[k] = pl->sendbuf[k];
    }
    return ORC_OK;
}

/* y_L = A_L x_L for rank p (p = -1: every rank), written into y. */
int orc_local(orc_plan *pl, int p, const double *x, double *y)
{
    if (p < -1 || p >= pl->P) return ORC_EINVAL;
    for (int d = 0; d < pl->P; d++) {
        if (p >= 0 && d != p) continue;
        const orc_rank *r = &pl->rk[d];
        const double *xl = x + pl->bounds[d];
        double *yl = y + pl->bounds[d];
        for (int64_t i = 0; i < r->rows; i++) {
            double s = 0.0;
            for (int64_t k = r->l_ptr[i]; k < r->l_ptr[i + 1]; k++)
                s += r->l_val[k] * xl[r->l_col[k]];
            yl[i] = s;
        }
    }
    return ORC_OK;
}

/* y += y_R with y_R = A_R x_R for rank p (p = -1: every rank); x_R is p's
 * part of the receive buffer.  Rows without remote entries are untouched. */
int orc_remote(orc_plan *pl, int p, double *y)
{
    if (p < -1 || p >= pl->P) return ORC_EINVAL;
    for (int d = 0; d < pl->P; d++) {
        if (p >= 0 && d != p) continue;
        const orc_rank *r = &pl->rk[d];
        const double *xr = pl->recvbuf + pl->halo_off[d];
        double *yl = y + pl->bounds[d];
        for (int64_t i = 0; i < r->rows; i++) {
            if (r->r_ptr[i + 1] == r->r_ptr[i]) continue;
            double s = 0.0;
            for (int64_t k = r->r_ptr[i]; k < r->r_ptr[i + 1]; k++)
                s += r->r_val[k] * xr[r->r_col[k]];
            pl->yr[i] = s;
            yl[i] = yl[i] + pl->yr[i];
        }
    }
    return ORC_OK;
}

/* The whole product in the order the DAG fixes for one rank: pack, local,
 * copy, remote (one valid traversal). */
int orc_partitioned_spmv(orc_plan *pl, const double *x, double *y)
{
    int rc;
    if ((rc = orc_pack(pl, -1, x))) return rc;
    if ((rc = orc_local(pl, -1, x, y))) return rc;
    if ((rc = orc_copy(pl, -1))) return rc;
    return orc_remote(pl, -1, y);
}

/* Clear both halo buffers (used by tests that check an out-of-order
 * schedule really reads stale data). */
void orc_clear_buffers(orc_plan *pl)
{
    memset(pl->sendbuf, 0, (size_t)pl->n_send * sizeof(double));
    memset(pl->recvbuf, 0, (size_t)pl->n_send * sizeof(double));
}

/* ------------------------------------------------------------------ */
/* Plan export, for bit-exact comparisons.                              */
/* ------------------------------------------------------------------ */
enum {
    ORC_BOUNDS = 0,     /* int64[P+1] */
    ORC_L_PTR = 1,      /* int64[rows_p+1] */
    ORC_L_COL = 2,      /* int32[l_nnz_p] */
    ORC_L_VAL = 3,      /* double[l_nnz_p] */
    ORC_R_PTR = 4,      /* int64[rows_p+1] */
    ORC_R_COL = 5,      /* int32[r_nnz_p] */
    ORC_R_VAL = 6,      /* double[r_nnz_p] */
    ORC_HALO = 7,       /* int32[n_halo_p] */
    ORC_SEND_IDX = 8,   /* int32[n_send] */
    ORC_HALO_OFF = 9,   /* int64[P+1] */
    ORC_SEG_OFF = 10,   /* int64[P*P+1] */
    ORC_SENDBUF = 11,   /* double[n_send] */
    ORC_RECVBUF = 12    /* double[n_send] */
};

static int64_t export_len(const orc_plan *pl, int what, int p, size_t *elt,
                          const void **src)
{
    const orc_rank *r = (p >= 0 && p < pl->P) ? &pl->rk[p] : NULL;
    switch (what) {
    case ORC_BOUNDS: *elt = 8; *src = pl->bounds; return pl->P + 1;
    case ORC_SEND_IDX: *elt = 4; *src = pl->send_idx; return pl->n_send;
    case ORC_HALO_OFF: *elt = 8; *src = pl->halo_off; return pl->P + 1;
    case ORC_SEG_OFF: *elt = 8; *src = pl->seg_off; return (int64_t)pl->P * pl->P + 1;
    case ORC_SENDBUF: *elt = 8; *src = pl->sendbuf; return pl->n_send;
    case ORC_RECVBUF: *elt = 8; *src = pl->recvbuf; return pl->n_send;
    default: break;
    }
    if (!r) return -1;
    switch (what) {
    case ORC_L_PTR: *elt = 8; *src = r->l_ptr; return r->rows + 1;
    case ORC_L_COL: *elt = 4; *src = r->l_col; return r->l_nnz;
    case ORC_L_VAL: *elt = 8; *src = r->l_val; return r->l_nnz;
    case ORC_R_PTR: *elt = 8; *src = r->r_ptr; return r->rows + 1;
    case ORC_R_COL: *elt = 4; *src = r->r_col; return r->r_nnz;
    case ORC_R_VAL: *elt = 8; *src = r->r_val; return r->r_nnz;
    case ORC_HALO: *elt = 4; *src = r->halo; return r->n_halo;
    default: return -1;
    }
}

/* Number of elements of array `what` (for rank p where it is per rank). */
int64_t orc_plan_len(const orc_plan *pl, int what, int p)
{
    size_t elt;
    const void *src;
    return export_len(pl, what, p, &elt, &src);
}

int orc_plan_export(const orc_plan *pl, int what, int p, void *dst, int64_t cap)
{
    size_t elt;
    const void *src;
    int64_t len = export_len(pl, what, p, &elt, &src);
    if (len < 0 || len > cap) return ORC_EINVAL;
    if (len) memcpy(dst, src, (size_t)len * elt);
    return ORC_OK;
}
