/*
 * spmv.h -- C ABI of the row-partitioned FP64 SpMV operation DAG.
 *
 * The operation is the distributed sparse matrix-vector product of
 * Pearson, Javeed and Devine, "Machine Learning for CUDA+MPI Design Rules",
 * Sec. III-A and Fig. 3: contiguous, even row blocks of A, x and y are owned
 * by P ranks; rank p computes y_p = A_L x_L + A_R x_R, where A_L holds the
 * columns of its own block, A_R the rest, and x_R is assembled from the x
 * entries other ranks pack and send.  Here the P ranks are virtual ranks
 * sharing one GPU, and the exchange is a device-to-device copy.
 *
 * The four operations of Fig. 3c, with their dependencies (the DAG G_P):
 *   PACK   -> COPY       sendbuf[k] = x[send_idx[k]]  (Pack vertex)
 *   COPY   -> REMOTE     recvbuf <- sendbuf           (PostSends/PostRecvs/Wait*)
 *   LOCAL  -> REMOTE     y_p = A_L,p x_L              (y_L vertex)
 *                        y_p += A_R,p x_R             (y_R vertex)
 * A schedule is a topological order of the operations plus a map of each
 * operation to a stream (Sec. III-B, Eq. 1); synchronisation is inserted as
 * Table III prescribes.
 *
 * Conventions for every entry point:
 *   - Returns an spmv_status; never throws.  On failure a message is stored
 *     per thread and returned by spmv_last_error().
 *   - Device pointers (suffix _dev) are caller-owned, on the current device,
 *     and must stay valid until the work issued on the given stream ends.
 *     Host pointers (suffix _host) are read or written before return, unless
 *     stated otherwise.
 *   - Work is asynchronous on the given stream(s); no hidden synchronisation
 *     except in spmv_part_create, spmv_part_destroy, spmv_part_export_plan,
 *     spmv_part_query(SPMV_Q_ERROR), spmv_part_set_variant and
 *     spmv_part_set_op_variant (which may build a layout), the _host entry
 *     points, spmv_csr_error, spmv_batch_create / destroy / set_lanes and
 *     the serving entry points other than spmv_serve_single.
 *   - A plan computes one product at a time: its send and receive buffers
 *     are shared by all of its launches, so two executions of the same plan
 *     must not overlap on the GPU.  Different plans are independent.
 *   - Indices: column indices are int32 and n < 2^31; the number of nonzeros
 *     must also be below 2^31.
 *   - All FP values and accumulations are IEEE binary64.
 *   - Consecutive kernels of the operations on one stream are launched with
 *     programmatic dependent launch: a kernel may be scheduled as the
 *     previous one's CTAs exit and waits for its completion before touching
 *     memory, so ordering is unchanged.  SPMV_NO_PDL=1 in the environment
 *     (read once per process) launches them plainly.
 */
#ifndef SPMV_H
#define SPMV_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPMV_OK = 0,
    SPMV_EINVAL = -1,    /* bad argument (size, pointer, selector, CSR) */
    SPMV_ENOMEM = -2,    /* a device or host allocation failed */
    SPMV_ECUDA = -3,     /* a CUDA runtime call failed */
    SPMV_ESCHED = -4,    /* schedule rejected: not a topological order, or a
                            stream id out of range; nothing was launched */
    SPMV_EBOUNDS = -5,   /* a size exceeds a fixed limit of the library */
    SPMV_ETIMEOUT = -6   /* a bounded device wait gave up (see SPMV_Q_ERROR) */
} spmv_status;

/* Operation kinds; op id = part * 4 + kind for the coarse (part 0) and
 * per-partition granularities; see SPMV_PER_SEGMENT for the third. */
enum { SPMV_OP_PACK = 0, SPMV_OP_LOCAL = 1, SPMV_OP_COPY = 2, SPMV_OP_REMOTE = 3 };

/* Granularity of the operations (Sec. III-A: one Pack vertex for all
 * peers versus one per peer).
 *   SPMV_COARSE        4 ops, each over every rank.
 *   SPMV_PER_PARTITION 4P ops, op 4p + kind: PACK of source rank p, COPY
 *                      into destination p, LOCAL / REMOTE of rank p;
 *                      PACK_q -> COPY_p when q sends to p.
 *   SPMV_PER_SEGMENT   one PACK and one COPY per halo segment (destination
 *                      p, source q, nonempty; the per-direction halo ops of
 *                      a stencil): ops 2p = LOCAL_p, 2p+1 = REMOTE_p, then
 *                      2P + 2k = PACK and 2P + 2k + 1 = COPY of segment k,
 *                      segments destination-major then by source;
 *                      PACK_k -> COPY_k -> REMOTE_p, LOCAL_p -> REMOTE_p.
 * spmv_part_op_info decodes an op id in every granularity. */
enum { SPMV_COARSE = 0, SPMV_PER_PARTITION = 1, SPMV_PER_SEGMENT = 2 };

typedef struct spmv_part spmv_part;   /* opaque; owns all plan memory */

/*
 * Build the partition plan (Sec. III-A, Fig. 3b) of the n x n CSR matrix
 * (row_ptr[n+1] int64, col_idx[nnz] int32, vals[nnz] double, all HOST
 * memory, read during the call) over P row-block ranks with
 * r_p = floor(p n / P), and upload it to the current device.
 *   A_L,p : entries of rows r_p..r_{p+1} with column in the same range,
 *           columns rebased to the block (x_L = x + r_p);
 *   H_p   : the sorted distinct columns outside the range (x_R's entries);
 *   A_R,p : the other entries, columns renumbered to positions in H_p;
 *   send buffer: destination-major, then source rank, then ascending column,
 *           so destination p's part is x[H_p] and the exchange is one copy.
 * granularity selects SPMV_COARSE, SPMV_PER_PARTITION or SPMV_PER_SEGMENT
 * (above).  Columns within a row may come in any order
 * and may repeat; each entry is kept and summed in the order given.
 * Errors: SPMV_EINVAL for n < 0, P < 1, a decreasing row_ptr, a column out
 * of [0, n), or NULL pointers with n > 0; SPMV_EBOUNDS for n or nnz >=
 * 2^31; SPMV_ENOMEM / SPMV_ECUDA.  *out is NULL on failure.
 */
int spmv_part_create(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                     const double* vals, int P, int granularity, spmv_part** out);

/* Synchronises the device, releases every graph, event and buffer. NULL ok. */
int spmv_part_destroy(spmv_part* part);

/* Scalar queries; `part_idx` selects a rank where the quantity is per rank
 * (ignored otherwise). */
enum {
    SPMV_Q_N = 0, SPMV_Q_P = 1, SPMV_Q_GRANULARITY = 2,
    SPMV_Q_NNZ = 3, SPMV_Q_NNZ_LOCAL = 4, SPMV_Q_NNZ_REMOTE = 5,
    SPMV_Q_N_SEND = 6,            /* total send-buffer entries */
    SPMV_Q_N_HALO = 7,            /* |H_p| of rank part_idx */
    SPMV_Q_N_REMOTE_ROWS = 8,     /* rows with at least one remote entry */
    SPMV_Q_N_OPS = 9,             /* operations of the DAG */
    SPMV_Q_N_EDGES = 10,          /* dependency edges of the DAG */
    SPMV_Q_ALG_BYTES = 11,        /* algorithmic bytes of one SpMV: the LOCAL
                                     op's, plus 12 per remote entry, 8 per
                                     compressed remote row (row id, pointer)
                                     and 4 for the closing pointer, 16 per
                                     remote row (y read and written),
                                     12 per send slot (index, slot), 16 per
                                     exchanged entry, 8 per remote halo read */
    SPMV_Q_ALG_BYTES_LOCAL = 12,  /* algorithmic bytes of the LOCAL op: 12 per
                                     local entry (value, column), 4 per row
                                     pointer (n + 1), 16 per row (x, y) */
    SPMV_Q_DEVICE_BYTES = 13,     /* device memory the plan holds */
    SPMV_Q_LAST_RECORDS = 14,     /* events recorded for DAG edges by the last issue */
    SPMV_Q_LAST_WAITS = 15,       /* stream waits issued for DAG edges by the last issue */
    SPMV_Q_ERROR = 16,            /* device error word (0 = none); synchronises */
    SPMV_Q_LOCAL_VARIANT = 17,
    SPMV_Q_N_LOCAL_TILES = 18,
    SPMV_Q_LAST_LAUNCHES = 19,    /* kernels launched by the last issue */
    SPMV_Q_REMOTE_VARIANT = 20,   /* 100 * variant + param of the REMOTE product
                                     (SPMV_Q_LOCAL_VARIANT: of the LOCAL one) */
    SPMV_Q_SELL_ENTRIES = 21,     /* padded entries of the sliced layout, local
                                     plus remote (0 until SELL is first set) */
    SPMV_Q_LAST_DEFERRED = 22     /* remote products the last spmv_schedule_run
                                     issued with a deferred wait (SPMV_RUN_DEFER) */
};
int spmv_part_query(const spmv_part* part, int what, int part_idx, int64_t* out);

/* Plan arrays for bit-exact comparisons, copied back from the DEVICE copy
 * the kernels use, in canonical per-rank form. */
enum {
    SPMV_X_BOUNDS = 0,     /* int64[P+1]   row bounds r_p */
    SPMV_X_L_PTR = 1,      /* int64[rows_p+1] local row pointer from 0 (rank) */
    SPMV_X_L_COL = 2,      /* int32 rebased local columns (rank) */
    SPMV_X_L_VAL = 3,      /* double local values (rank) */
    SPMV_X_R_PTR = 4,      /* int64[rows_p+1] remote row pointer from 0 (rank) */
    SPMV_X_R_COL = 5,      /* int32 positions in H_p (rank) */
    SPMV_X_R_VAL = 6,      /* double remote values (rank) */
    SPMV_X_HALO = 7,       /* int32 H_p (rank) */
    SPMV_X_SEND_IDX = 8,   /* int32[n_send] x index of each send slot */
    SPMV_X_HALO_OFF = 9,   /* int64[P+1] start of destination p's part */
    SPMV_X_SEG_OFF = 10,   /* int64[P*P+1] start of segment (dst p, src q) at p*P+q */
    SPMV_X_SENDBUF = 11,   /* double[n_send] current send buffer */
    SPMV_X_RECVBUF = 12    /* double[n_send] current receive buffer */
};
/* Element count of array `what` (for rank part_idx where per rank), or < 0. */
int64_t spmv_part_export_len(const spmv_part* part, int what, int part_idx);
/* Copy array `what` to host_dst (capacity cap elements); synchronises.  The
 * matrix arrays of a plan whose CSR copy was released are exported after
 * rebuilding it (spmv_part_release_csr). */
int spmv_part_export_plan(const spmv_part* part, int what, int part_idx,
                          void* host_dst, int64_t cap);

/* Op id -> kind (SPMV_OP_*), destination rank and source rank (-1 where
 * the op has none: a coarse op, a per-partition PACK's destination, ...). */
int spmv_part_op_info(const spmv_part* part, int op, int32_t* kind, int32_t* dst, int32_t* src);

/* DAG of the plan's operations as (src op, dst op) int32 pairs. */
int spmv_part_dag(const spmv_part* part, int32_t* edges_host, int64_t cap_pairs,
                  int64_t* n_pairs_out);

/* Kernel variant of the LOCAL and REMOTE products (every variant gives the
 * same y within the FP64 bound; each is deterministic on its own).
 *   TILE   param = geometry 0..4: rows staged in shared memory by bulk
 *          copies, 1 or 2 threads per row (the geometry fixes which)
 *   VECTOR param = lanes per row (2..32), 4 entries per lane per step with
 *          128-bit loads
 *   PAIRS  param = lanes per row (1, 2, 4, 8), one aligned pair of entries per
 *          lane per step, FMA count = the warp's longest share; 102 / 104:
 *          2 / 4 lanes with fewer pairs in flight and 8 CTAs per SM
 *   MERGE  merge-path split with deterministic carries (param ignored)
 *   WARP   param = geometry 0..4: warp-private shared-memory pipelines of
 *          32-row tiles (bulk copies per warp, no block-wide barrier), one
 *          thread per row, one DFMA per entry
 *   SELL   param = 4, 8, 9 (entries per lane per step; 8, 4 and 4 CTAs per
 *          SM) or 104 / 105 / 106 / 107 (4 at 6, 8 at 5, 8 at 6, 9 at 5 CTAs
 *          per SM, in fewer registers), each + 2000 (2004, ..., 2107) for the same
 *          launch with the work units cut into contiguous ranges of equal
 *          estimated cost, one per CTA, instead of dealt round-robin to the
 *          warps (evens out the SMs on skewed rows; y is the same bit for
 *          bit; the ranges are built when the variant is set, for every
 *          rank and for all ranks).  A sliced-ELL copy of A_L and A_R that the plan builds
 *          on first use and holds until destroyed.  Per rank, rows longer
 *          than 64 entries are summed by a whole warp each; the others sit
 *          in slices of 32 positions (entry j of position r at slice offset
 *          + 32 j + r, padded to the slice's longest row with value 0 and
 *          column 0), in natural row order when that pads by at most 1/8
 *          (+1024 entries), else sorted by length.  One thread per short
 *          row, one FMA per stored entry in storage order (padded slots
 *          discarded), so y equals WARP's bit for bit on matrices without
 *          long rows.  SPMV_EBOUNDS beyond 2^31 padded entries.
 *   SELL16 the SELL layout of the LOCAL product with each slot's column
 *          stored as a 16-bit delta to its row (x index = row + delta):
 *          10 instead of 12 bytes per slot.  LOCAL only, through
 *          spmv_part_set_op_variant; SPMV_EINVAL (nothing changed) when a
 *          local column lies more than 32767 rows from its row, or for the
 *          REMOTE product.  Same y as SELL, bit for bit.
 * Fails with SPMV_EINVAL while captured graphs exist (they hold the old
 * kernels' tables). */
enum {
    SPMV_VARIANT_TILE = 0,
    SPMV_VARIANT_VECTOR = 1,
    SPMV_VARIANT_MERGE = 2,
    SPMV_VARIANT_PAIRS = 3,
    SPMV_VARIANT_WARP = 4,
    SPMV_VARIANT_SELL = 5,
    SPMV_VARIANT_SELL16 = 6
};
/* Sets the variant of both products. */
int spmv_part_set_variant(spmv_part* part, int variant, int param);
/* Sets the variant of one product: op_kind SPMV_OP_LOCAL or SPMV_OP_REMOTE. */
int spmv_part_set_op_variant(spmv_part* part, int op_kind, int variant, int param);

/*
 * Release the plan's CSR copy of the matrix once both products use the
 * sliced layout (LOCAL SPMV_VARIANT_SELL or SELL16, REMOTE SELL): that
 * layout is a second copy of every entry, so the plan otherwise holds the
 * matrix twice.  The entries of rows longer than 64 (which the sliced
 * products read from the CSR) move to compact arrays of their own; then the
 * CSR columns and values of A_L and A_R are freed, and A_L's 32-bit slot
 * columns too while its product uses the 16-bit deltas.  Row pointers stay.
 * Products give the same y, bit for bit.  Whatever needs the CSR again
 * (selecting a non-sliced variant, or the 32-bit LOCAL one after SELL16;
 * spmv_part_export_plan of SPMV_X_L_COL / L_VAL / R_COL / R_VAL;
 * spmv_part_check) first rebuilds it on the device from the sliced layout
 * and keeps it.  SPMV_Q_DEVICE_BYTES reports the memory held.  Synchronises.
 * Errors: SPMV_EINVAL when a product does not use the sliced layout or while
 * captured graphs exist; a no-op if already released.
 */
int spmv_part_release_csr(spmv_part* part);

/*
 * The four operations (Fig. 3c).  `part_idx` = -1 runs the op for every
 * rank in one launch (coarse); 0 <= part_idx < P runs rank part_idx's op.
 *   spmv_pack:      sendbuf slots owned by source rank part_idx <- x
 *   spmv_local:     y rows of rank part_idx <- A_L x_L (overwrites)
 *   spmv_halo_copy: destination part_idx's slice of recvbuf <- sendbuf
 *   spmv_remote:    y rows of rank part_idx with remote entries += A_R x_R
 * x_dev / y_dev: n doubles on the device (caller-owned).
 */
int spmv_pack(spmv_part* part, int part_idx, const double* x_dev, cudaStream_t s);
int spmv_local(spmv_part* part, int part_idx, const double* x_dev, double* y_dev,
               cudaStream_t s);
int spmv_halo_copy(spmv_part* part, int part_idx, cudaStream_t s);
int spmv_remote(spmv_part* part, int part_idx, double* y_dev, cudaStream_t s);

/*
 * Run one implementation (Sec. III-B): op_order[n_ops] is a permutation of
 * the op ids, stream_of_op[op id] in [0, n_streams) binds each op to
 * streams[..].  Before anything is launched the order is checked to be
 * topological for the DAG and every stream id to be in range (else
 * SPMV_ESCHED).  Issue follows Table III: an op waits (cudaStreamWaitEvent)
 * on an event recorded right after each predecessor bound to another
 * stream, and nothing for a predecessor on its own stream.  The artificial
 * start and end vertices are a fork from streams[0] to every other used
 * stream and a join of all of them back into streams[0], so back-to-back
 * runs never overlap.
 * flags: SPMV_RUN_EAGER issues the ops now, in order.
 *        SPMV_RUN_CAPTURE captures the same issue into a CUDA graph started
 *          on streams[0], instantiates it and returns its handle in
 *          *graph_handle_inout (nothing runs).  x_dev and y_dev are baked in.
 *        SPMV_RUN_REPLAY launches graph *graph_handle_inout on streams[0];
 *          x_dev / y_dev must equal the captured ones (else SPMV_EINVAL).
 * A graph keeps only dependencies, so two orders that differ only in the
 * relative order of ops on different streams give the same graph.
 * SPMV_RUN_RELAXED (or-ed into CAPTURE; SPMV_EINVAL with EAGER; ignored by
 *   REPLAY) lets an op with no DAG predecessor (a pack or a local product)
 *   overlap the kernel before it on its stream: it does not wait for that
 *   kernel, which releases it as its CTAs start (programmatic dependent
 *   launch without the wait), so it fills that kernel's tail.  Every other
 *   op still waits for the kernels it depends on, and every DAG edge, also
 *   between two ops of one stream, becomes an event.  An extension, not the
 *   paper's stream semantics (where the kernels of a stream run one after
 *   another, the default here).  Ops of one product touch common data only
 *   along DAG edges, so y is the same, bit for bit.
 * SPMV_RUN_DEFER (or-ed into CAPTURE, alone or with SPMV_RUN_RELAXED;
 *   SPMV_EINVAL with EAGER; ignored by REPLAY) keeps the stream semantics
 *   above but lets a remote product in the sliced layout (SPMV_VARIANT_SELL)
 *   start while the kernel before it on its stream runs, when that kernel
 *   writes none of the product's inputs but y (any op that is not the
 *   product's DAG predecessor, or its local product): the product reads
 *   A_R and the halo and sums its rows first, and waits for that kernel
 *   only before it adds the sums into y, so the remote product overlaps
 *   the tail of, say, the local product of its rank.  The kernel before it
 *   releases it as its CTAs start.  The product's edges from other streams
 *   stay full dependencies in the graph (checked after capture).  An
 *   extension of the paper's stream semantics; y is the same, bit for bit.
 */
enum { SPMV_RUN_EAGER = 0, SPMV_RUN_CAPTURE = 1, SPMV_RUN_REPLAY = 2, SPMV_RUN_RELAXED = 4, SPMV_RUN_DEFER = 8 };
int spmv_schedule_run(spmv_part* part, const int32_t* op_order,
                      const int32_t* stream_of_op, int n_ops,
                      cudaStream_t* streams, int n_streams,
                      const double* x_dev, double* y_dev,
                      int flags, int64_t* graph_handle_inout);

/* Release one captured graph (handle from SPMV_RUN_CAPTURE). */
int spmv_graph_destroy(spmv_part* part, int64_t graph_handle);

/*
 * End-to-end product through host buffers: copies x_host (n doubles,
 * should be pinned) into a plan-owned device vector, replays graph
 * `graph_handle` (captured with spmv_part_io_buffers' vectors) on stream s,
 * and copies y back into y_host; returns after the stream finished.
 */
int spmv_part_io_buffers(spmv_part* part, double** x_dev_out, double** y_dev_out);
int spmv_apply_host(spmv_part* part, int64_t graph_handle, const double* x_host,
                    double* y_host, cudaStream_t s);
/*
 * The same end-to-end product with the transfers overlapped: x_host's row
 * blocks are copied in one by one on copy_stream, rank p's LOCAL product
 * starts as soon as block p has arrived (it reads no other x), on
 * compute_stream for even p and on a plan-owned second stream for odd p (so
 * consecutive ranks' launches overlap); PACK and COPY for every rank run on
 * a third plan-owned stream once all of x has arrived; each rank's REMOTE
 * product follows its LOCAL product (same stream) once COPY is done.
 * y comes back in two parts on a plan-owned stream of its own (so the copies
 * out overlap the copies in, the link's two directions): each rank's longest
 * run of rows without remote entries as soon as its LOCAL product is done
 * (those rows are final then), its other rows after its REMOTE product.  Returns
 * after y has arrived.  The two streams must differ.  Same y as the graph
 * path, bit for bit (the same kernels on the same rows).  Plan-owned device
 * vectors as above.
 */
int spmv_apply_host_pipelined(spmv_part* part, const double* x_host, double* y_host,
                              cudaStream_t copy_stream, cudaStream_t compute_stream);
/*
 * A stream of independent end-to-end products y_k = A x_k, k = 0 .. count-1,
 * through host buffers (the host-buffer form of a batch of right-hand sides
 * that arrive one after another; each product as in
 * spmv_apply_host_pipelined, §III-A's four operations per product).
 *   x_k = x_host + k * x_stride, y_k = y_host + k * y_stride (strides in
 *   doubles, >= 0; x_stride 0 sends the same host vector every time, y_stride
 *   0 lets every product write the same host vector, the last one's result
 *   staying; otherwise y_stride >= n).  Host vectors should be pinned.
 *   Overlap: the products alternate between two plan-owned pairs of device
 *   vectors, so product k+1's x goes in while product k computes and its y
 *   goes out: the link carries both directions at once.  Product k+1's
 *   copies in wait until product k-1's readers of that x are done, its
 *   products until product k-1's y has gone out, and its exchange until
 *   product k's REMOTE products have read the receive buffer; nothing else
 *   is shared.  Each y_k is the same, bit for bit, as
 *   spmv_apply_host_pipelined's for x_k.
 *   flags: SPMV_HOST_X_BLOCKS sends x rank block by rank block, each rank's
 *   LOCAL product starting once its block is in (else x goes in one copy);
 *   SPMV_HOST_Y_PARTS returns each rank's rows as soon as they are final, as
 *   spmv_apply_host_pipelined does (else y comes back in one copy after the
 *   last REMOTE product).  Both set is spmv_apply_host_pipelined's order;
 *   every copy costs a few microseconds beyond its bytes, so in a stream of
 *   products, where the next product's transfers already fill the link,
 *   fewer copies can be faster.  The results do not depend on the flags.
 *   Streams: as spmv_apply_host_pipelined (the two must differ).  Returns
 *   after every y_k has arrived.  The second pair of device vectors (16 n
 *   bytes) is allocated by the first call and kept with the plan.
 *   Errors: SPMV_EINVAL (count or a stride negative, NULL host buffers,
 *   equal streams, 0 < y_stride < n with count > 1, unknown flags),
 *   SPMV_ENOMEM, SPMV_ECUDA.
 */
enum { SPMV_HOST_X_BLOCKS = 1, SPMV_HOST_Y_PARTS = 2 };
int spmv_apply_host_many(spmv_part* part, int64_t count, const double* x_host, int64_t x_stride,
                         double* y_host, int64_t y_stride, int flags, cudaStream_t copy_stream,
                         cudaStream_t compute_stream);

/*
 * Plain CSR product y = A x on caller-owned DEVICE arrays with the
 * merge-path kernel (equal work per CTA whatever the row lengths; rows cut
 * between threads or CTAs are finished in a fixed order, so y is
 * deterministic).  row_ptr_dev: int32[n+1] with row_ptr[0] = 0 and
 * row_ptr[n] = nnz, non-decreasing; col_idx_dev: int32[nnz] in [0, n);
 * vals_dev: double[nnz]; x_dev, y_dev: double[n]; every array 16-byte
 * aligned.  The arrays are read only inside their bounds.  Scratch: 48 bytes
 * per 2048 merge items (rows + entries), taken with cudaMallocAsync on s and
 * released with cudaFreeAsync on s.  Preconditions on the CSR contents are
 * the caller's: they are not checked on the device.
 * Errors: SPMV_EINVAL (sizes, NULL or misaligned pointers), SPMV_EBOUNDS
 * (n + nnz >= 2^31 - 2048), SPMV_ENOMEM, SPMV_ECUDA.  A bounded device
 * wait that gives up is reported by spmv_csr_error.
 */
int spmv_csr_merge(int64_t n, int64_t nnz, const int32_t* row_ptr_dev,
                   const int32_t* col_idx_dev, const double* vals_dev,
                   const double* x_dev, double* y_dev, cudaStream_t s);

/*
 * spmv_csr_merge without any allocation: the same product, kernels and
 * result as spmv_csr_merge, with its scratch (tile coordinates and row
 * carries) in a fixed array compiled into the library instead of memory
 * taken at call time.  The paper has no counterpart; this entry point is for
 * callers that must not allocate device memory during a call: code that
 * runs inside a host application owning every device allocation through its
 * own fixed pool, latency-bound loops where an allocation may synchronise
 * or grow a pool at an unpredictable moment, and work recorded into a CUDA
 * graph whose owner does not accept memory-allocation nodes.
 *   Limit: n + nnz <= 134 217 728 (65 536 tiles of 2048 merge items); larger
 *   inputs fail with SPMV_EBOUNDS before anything is launched.  The array
 *   takes 3 MiB on every GPU that loads the library, until the process exits.
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Sharing: every call on a device uses the same array.  Each call rewrites
 *   the part it reads before reading it, so leftovers of an earlier call are
 *   never used, but calls whose work overlaps on the GPU (other streams, or
 *   other host threads) race on the array and must be serialised by the
 *   caller.
 * Arguments, alignment, preconditions and other errors as spmv_csr_merge.
 * Calls no cudaMalloc, cudaFree or allocating library routine.
 */
int spmv_csr_merge_noalloc(int64_t n, int64_t nnz, const int32_t* row_ptr_dev,
                           const int32_t* col_idx_dev, const double* vals_dev,
                           const double* x_dev, double* y_dev, cudaStream_t s);

/* Device error word of the plan-free entry points on the current device
 * (0 = none; SPMV_ETIMEOUT's magnitude after a bounded wait gave up); reads
 * and clears it, synchronising the device. */
int spmv_csr_error(int64_t* out);

/*
 * Batched products: many independent CSR matrices (no partitioning) kept
 * resident in HBM and multiplied in one persistent launch per layout
 * (CSR modes, sliced layout).  Work items are blocks of up to 256 rows of
 * one matrix (CSR modes) or up to 8 slices or 32 long rows of one matrix
 * (sliced layout), claimed by warps through an atomic ticket, matrix by
 * matrix with each matrix's heaviest items first; each row is summed by
 * `lanes` lanes (set per matrix, e.g. by an autotuner), a row longer than
 * 64 entries by a whole warp, in a fixed order, so y is the same, bit for
 * bit, as with spmv_batch_run_separate, which launches the same row code
 * once per matrix.  Not part of the paper's method: a way of running many
 * of its SpMVs at once.
 * spmv_batch_create: `count` matrices given as HOST CSR arrays (n[m],
 *   row_ptr[m][n[m]+1] int64, col_idx[m] int32 in [0, n[m]), vals[m]),
 *   copied to the current device.  Errors as spmv_part_create.
 * x_dev / y_dev: the concatenation of every matrix's x / y; matrix m's part
 *   starts at spmv_batch_query(SPMV_BQ_OFFSET, m).
 */
typedef struct spmv_batch spmv_batch;
enum {
    SPMV_BQ_COUNT = 0, SPMV_BQ_TOTAL_ROWS = 1, SPMV_BQ_TOTAL_NNZ = 2, SPMV_BQ_ITEMS = 3,
    SPMV_BQ_ALG_BYTES = 4,   /* 12 B/entry + 4 B/row pointer + 16 B/row (x read, y written) */
    SPMV_BQ_OFFSET = 5, SPMV_BQ_N = 6, SPMV_BQ_NNZ = 7, SPMV_BQ_LANES = 8,  /* of matrix m */
    SPMV_BQ_DEVICE_BYTES = 9,  /* device memory the batch holds */
    SPMV_BQ_LAUNCHES = 10      /* kernels one spmv_batch_run launches (0-2) */
};
int spmv_batch_create(int count, const int64_t* n, const int64_t* const* row_ptr,
                      const int32_t* const* col_idx, const double* const* vals,
                      spmv_batch** out);
int spmv_batch_destroy(spmv_batch* batch);
/* Lanes per row (1, 2, 4, 8, 16, 32) of matrix m, or of every matrix (m = -1);
 * 0 selects warp-staged rows (each warp stages its 32 rows' entries in shared
 * memory and sums one row per lane; for short rows); SPMV_BATCH_SLICED (64)
 * a sliced layout built on first use (a second copy of the matrix in device
 * memory): slices of 32 rows, one row per lane, entry j of lane r at
 * slice offset + 32 j + r, rows padded to the slice's longest with value 0;
 * natural row order when that pads by at most 1/8 and no row exceeds 64
 * entries, else rows sorted by length with the longer-than-64 rows summed
 * by whole warps.  Synchronises the device (no launch of the batch may be
 * in flight). */
enum { SPMV_BATCH_SLICED = 64 };
int spmv_batch_set_lanes(spmv_batch* batch, int m, int lanes);
int spmv_batch_query(const spmv_batch* batch, int what, int m, int64_t* out);
/* Every product on stream s: one persistent launch over the sliced-layout
 * matrices and one over the others (either left out when it has no work). */
int spmv_batch_run(spmv_batch* batch, const double* x_dev, double* y_dev, cudaStream_t s);
/* End to end through HOST buffers (x_host, y_host: the concatenated vectors,
 * pinned for full speed): the matrices are cut into `chunks` (1..64) runs of
 * whole matrices with about equal rows; chunk c's x is copied in on s_in,
 * its products run on s_compute once it has arrived (the persistent kernels
 * of spmv_batch_run over the chunk's items, so the same y bit for bit), and
 * its y is copied out on s_out while later chunks
 * are still in flight.  The three streams must differ.  Returns after y has
 * arrived.  Uses batch-owned device vectors (allocated on first use). */
int spmv_batch_run_host(spmv_batch* batch, const double* x_host, double* y_host, int chunks,
                        cudaStream_t s_in, cudaStream_t s_compute, cudaStream_t s_out);
/* A stream of independent batched products through host buffers: product
 * k reads x_host + k * x_stride and writes y_host + k * y_stride (strides in
 * doubles over the batch's concatenated rows, >= 0; 0 reuses one host
 * vector, the last product's y staying; otherwise y_stride >= the total
 * rows), each in `chunks` chunks as spmv_batch_run_host.  Consecutive
 * products alternate between two batch-owned pairs of device vectors, so
 * product k+1's x goes in while product k computes and its y comes back;
 * product k+1's copies in wait for the products that read that pair's x
 * (product k-1), its products for that pair's y to have gone out.  Each y_k
 * is bit for bit spmv_batch_run_host's.  Returns after every y_k arrived.
 * Errors: SPMV_EINVAL (negative count or stride, NULL host buffers, chunks
 * outside [1, 64], equal streams, overlapping y strides), SPMV_ENOMEM,
 * SPMV_ECUDA. */
int spmv_batch_run_host_many(spmv_batch* batch, int64_t count, const double* x_host, int64_t x_stride,
                             double* y_host, int64_t y_stride, int chunks, cudaStream_t s_in,
                             cudaStream_t s_compute, cudaStream_t s_out);
/* Release the batch's CSR copy once every matrix uses the sliced layout
 * (SPMV_BATCH_SLICED), which is a second copy of every entry: only the rows
 * longer than 64 entries (which the sliced products, batched and served,
 * read from the CSR) stay, in compact arrays.  Results are unchanged, bit for
 * bit.  Setting any matrix to a non-sliced layout afterwards first rebuilds the
 * full CSR on the device (from the sliced layout and the kept long rows).  A
 * server created while the CSR is released serves the sliced layout only.
 * Synchronises.  SPMV_EINVAL while a matrix is not sliced; a no-op if already
 * released.  SPMV_BQ_DEVICE_BYTES reports the memory held. */
int spmv_batch_release_csr(spmv_batch* batch);
/* The same products as one launch per matrix (only matrix m if m >= 0). */
int spmv_batch_run_separate(spmv_batch* batch, int m, const double* x_dev, double* y_dev,
                            cudaStream_t s);

/*
 * Serving: SpMV requests over the matrices of a resident batch, with
 * continuous batching.  A request names a matrix, a width k in 1..8 (right-
 * hand sides) and a 64-bit seed; its X (n x k) is drawn on the device: element
 * (i, j) is 2 u - 1 with u = (SplitMix64(seed, 8 i + j) >> 11) * 2^-53, where
 * SplitMix64(s, t) is the SplitMix64 output for state s + (t + 1) * golden
 * (Steele, Lea and Flood).  Not part of the paper's method: a serving loop
 * around its SpMV.
 * spmv_serve_create: n_streams (1..64) stream slots, one block in flight per
 *   slot; budget_bytes covers the resident matrices plus a pool from which
 *   every in-flight block of total width w takes 16 n w bytes (X and Y,
 *   n x w doubles each, row-major); SPMV_ENOMEM when the budget is below the
 *   resident matrices, SPMV_EBOUNDS for a matrix with n >= 2^28.
 * spmv_serve_run: runs n_req requests open loop against their arrival times
 *   (seconds from the call, non-decreasing), on the host thread, until all
 *   completed.  Queues are served oldest first (the matrix whose oldest
 *   waiting request arrived first; ties by request index).  BATCHED merges
 *   the oldest requests of one matrix into one block of total width <= 8
 *   whenever a slot and pool memory are free; requests arriving while blocks
 *   run join at the next turn of the loop.  When every matrix is in the
 *   sliced layout, BATCHED goes further: a free slot takes ceil(blocks /
 *   slots) of the blocks the queues would form (at most the group size,
 *   spmv_serve_set_group_max) and runs more than one, across matrices, as one
 *   group with one launch per kernel kind (X generation, slices, long rows);
 *   while no more blocks wait than there are slots every block thus gets a
 *   slot of its own, and groups grow only with a longer queue.
 *   PLAIN launches every request alone (one block per request).  Outputs:
 *   latency_s[r] = observed completion - arrival; hash_out[r] (optional) an
 *   order-independent 64-bit hash of the bits of request r's Y; stats (6
 *   int64, optional): blocks launched, most blocks in flight, launches that
 *   waited for pool memory, peak pool bytes, elapsed ns, requests admitted
 *   while blocks were in flight.  Each column of a block is summed in the
 *   same order whatever the block's partners, so Y (and the hash) of a
 *   request is the same alone and in any mix.  SPMV_ETIMEOUT if no request
 *   completes for 30 s after the last arrival; SPMV_ENOMEM (before any
 *   launch) when a width-8 block of any of the matrices exceeds the pool.
 * Rows are summed in length buckets fixed per matrix at creation (short rows
 * by 1-8 lanes chosen from the mean length, rows up to 256 entries by 8
 * lanes, longer rows by a whole warp), so skewed matrices keep warps busy;
 * a matrix whose batch layout is SPMV_BATCH_SLICED when a block is launched
 * is summed over that layout instead (one thread per row, its long rows by
 * whole warps).  Choose the layouts before creating the server: the budget
 * counts the batch's device memory at creation.
 * spmv_serve_single: one request alone on stream s into caller buffers
 *   x_dev, y_dev (n x width doubles each, row-major).
 */
typedef struct spmv_server spmv_server;
enum { SPMV_SERVE_BATCHED = 0, SPMV_SERVE_PLAIN = 1 };
int spmv_serve_create(spmv_batch* matrices, int n_streams, int64_t budget_bytes,
                      spmv_server** out);
int spmv_serve_destroy(spmv_server* server);
int spmv_serve_run(spmv_server* server, int64_t n_req, const int32_t* matrix,
                   const int32_t* width, const uint64_t* seed, const double* arrival_s,
                   int mode, double* latency_s, uint64_t* hash_out, int64_t* stats);
/* Most blocks a grouped launch takes (1..64, default 64): smaller groups
 * finish sooner, larger ones launch less.  SPMV_EINVAL outside the range. */
int spmv_serve_set_group_max(spmv_server* server, int max_blocks);
/* The bits of the binary64 value m * 2^-52 - 1 (the 2 u - 1 above, for the
 * 53-bit draw m = SplitMix64(...) >> 11; only the low 53 bits of m are read),
 * computed on the host by the integer construction the device generator runs.
 * Exact, so it equals converting m to double and subtracting 1; no GPU. */
uint64_t spmv_serve_pm1_bits(uint64_t m);
/* Kernels launched by the last spmv_serve_run (every block's X generator
 * and products). */
int spmv_serve_launches(const spmv_server* server, int64_t* out);
int spmv_serve_single(spmv_server* server, int matrix, int width, uint64_t seed,
                      double* y_dev, double* x_dev, cudaStream_t s);

/* Index check of a plan (a memory checker's job, done by the library): reads
 * every index array and counts into *bad_out the indices outside the range
 * the plan's definition allows (Sec. III-A): A_L's columns inside their
 * rank's block, A_R's receive-buffer positions inside their rank's halo, the
 * remote rows inside their rank's rows, every send slot of segment (p, q)
 * naming a row of q, the per-rank pack positions inside the send buffer,
 * row pointers ascending from 0 to the entry count, and, once built, every
 * live slot of the sliced layouts (and of the 16-bit deltas) inside x or the
 * receive buffer, with each long-row piece inside its row, and the y row the
 * remote layout stores for each of rank p's positions inside p's rows.  No index is used
 * to address memory, so a damaged plan is reported, not dereferenced.  0 for
 * every plan this library builds.  Synchronises. */
int spmv_part_check(spmv_part* part, int64_t* bad_out);
/* Self-test of those checks on a planted 3-row CSR and index list with one
 * out-of-range index each: *found_out receives 2.  Synchronises. */
int spmv_selftest_check(int64_t* found_out);

/* Self-test of the bounded device waits: one thread waits on an mbarrier
 * that nothing ever completes; the wait gives up after limit_ns (1e3..2e9)
 * and *status_out receives 6 (the magnitude of SPMV_ETIMEOUT) -- the status
 * every kernel of the library reports through its error word when a wait
 * runs out.  Synchronises; leaves the context usable. */
int spmv_selftest_wait_timeout(int64_t limit_ns, int64_t* status_out);

/* FP64 fused multiply-add throughput probe (a measurement helper, not part
 * of the paper's method): the second roofline of the product, whose cost on
 * this part is one DFMA per stored entry.  Launches SM count x ctas_per_sm
 * (1..8) CTAs of 256 threads on stream s; in every warp the first `lanes`
 * (1..32) lanes run 8 independent chains of `iters` DFMAs each; every thread
 * then writes one double to out_dev (caller-owned device memory of at least
 * out_cap >= SM count x ctas_per_sm x 256 doubles, 8-byte aligned).
 * *dfma_out receives the DFMAs the launch executes (lane operations; with
 * lanes < 32 the warp instructions number 32 / lanes times fewer per lane
 * operation).  Time it with events on s; asynchronous, no allocation.
 * Errors: SPMV_EINVAL for arguments out of range. */
int spmv_probe_dfma(int64_t iters, int ctas_per_sm, int lanes, double* out_dev, int64_t out_cap,
                    int64_t* dfma_out, cudaStream_t s);

/* Gather throughput probe (a measurement helper, not part of the paper's
 * method): the rate at which the GPU serves scattered 8-byte reads, the
 * bound of a product whose x entries are far apart (each costs its own
 * cache sector).  Launches SM count x ctas_per_sm (1..8) CTAs of 256 threads
 * on stream s; thread g of the T launched sums table_dev[idx_dev[k]] over
 * k = g, g + T, g + 2T, ... < count, four gathers in flight, and writes the
 * sum to out_dev[g].  table_dev: doubles (8-byte aligned); idx_dev: count
 * int32 positions into it (4-byte aligned), each must lie inside the table
 * (the caller's precondition, not checked); out_dev: at least out_cap >=
 * T doubles.  Time it with events on s; asynchronous, no allocation.
 * Errors: SPMV_EINVAL for arguments out of range. */
int spmv_probe_gather(const double* table_dev, const int32_t* idx_dev, int64_t count, int ctas_per_sm,
                      double* out_dev, int64_t out_cap, cudaStream_t s);

/* Test hook of the merge-path kernel's give-up path (the path a bounded wait
 * that runs out takes), for the plan-free entry points spmv_csr_merge and
 * spmv_csr_merge_noalloc: while set (tile >= 0), their launches treat merge
 * tile `tile` and every later tile as if the wait for its staged copy had run
 * out, once that copy has landed (so no copy is left in flight).  Such a
 * launch sets the error word (spmv_csr_error reports 6), leaves the rows of
 * the abandoned tiles unfinished, marks their carries empty and writes nothing
 * outside y[0, n).  tile = -1 turns the hook off (the default).  Process-wide;
 * plans are not affected.  SPMV_EINVAL outside [-1, 2^30). */
int spmv_selftest_merge_abort(int64_t tile);

/* Thread-local message describing the last failure of this thread. */
const char* spmv_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SPMV_H */
