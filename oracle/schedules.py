"""Schedule space of Sec. III-B / III-C, by brute force.

TEST INFRASTRUCTURE (part of the oracle; see ``oracle/__init__.py``).

An implementation of a program P is a topological traversal of its DAG G_P
(Sec. III-B, Eq. 1) in which every GPU vertex is bound to a stream
(Table II: GPU -> BoundGPU_s).  Two implementations that differ only by a
bijection of the streams are the same program and are pruned (Sec. III-C.2).
Synchronisation operations follow Table III.

Everything here is written the slow, obvious way: all permutations times all
stream maps, filtered.  It is meant for tiny DAGs only.

Canonical form chosen for the bijection pruning: streams are numbered in
order of first use along the traversal (the first GPU op is on stream 0 and
each op is on a stream already used or on the next unused number).
"""
import itertools

# ------------------------------------------------------------------ #
# DAGs                                                                 #
# ------------------------------------------------------------------ #
PACK, LOCAL, COPY, REMOTE = 0, 1, 2, 3
KIND_NAMES = ("pack", "local", "copy", "remote")


def coarse_dag():
    """The SpMV DAG with one vertex per operation, spanning every rank.

    Pack -> exchange (the packed values must exist before they are sent),
    exchange -> remote product (x_R must be assembled, Sec. III-A), and
    local product -> remote product (the remote product accumulates into
    the y the local product wrote).  Returns (ops, edges) with op ids
    0..3 = pack, local, copy, remote.
    """
    ops = [PACK, LOCAL, COPY, REMOTE]
    edges = [(PACK, COPY), (COPY, REMOTE), (LOCAL, REMOTE)]
    return ops, edges


def per_partition_dag(P, sends):
    """One vertex per operation per rank (the finer granularity of
    Sec. III-A).  ``sends(q, p)`` is true when rank q packs entries for
    rank p.  Op id = rank * 4 + kind."""
    ops = list(range(4 * P))
    edges = []
    for p in range(P):
        for q in range(P):
            if q != p and sends(q, p):
                edges.append((4 * q + PACK, 4 * p + COPY))
        edges.append((4 * p + COPY, 4 * p + REMOTE))
        edges.append((4 * p + LOCAL, 4 * p + REMOTE))
    return ops, edges


def per_segment_dag(P, sends):
    """One PACK and one COPY per halo segment (destination p, source q), the
    finer granularity the paper's future work names (per-peer operations,
    per-direction halos of a stencil).  Op ids: 2p = LOCAL of rank p,
    2p + 1 = REMOTE of rank p, then for the k-th segment in destination-major,
    source-minor order 2P + 2k = its PACK and 2P + 2k + 1 = its COPY.
    Returns (ops, edges, segments)."""
    segs = [(p, q) for p in range(P) for q in range(P) if q != p and sends(q, p)]
    ops = list(range(2 * P + 2 * len(segs)))
    edges = [(2 * p, 2 * p + 1) for p in range(P)]
    for k, (p, q) in enumerate(segs):
        edges.append((2 * P + 2 * k, 2 * P + 2 * k + 1))
        edges.append((2 * P + 2 * k + 1, 2 * p + 1))
    return ops, edges, segs


def paper_fig3c_dag():
    """A reading of the SpMV DAG of Fig. 3c, whose image is not available.

    The text names vertex 1 = start, 2 = Pack, 4 = PostSends,
    5 = PostRecvs; y_L, y_R, WaitSend, WaitRecv and the end vertex are named
    by the rules of Tables VI-VIII.  Reading used here:
      1 start, 2 Pack, 3 y_L, 4 PostSends, 5 PostRecvs, 6 WaitSend,
      7 WaitRecv, 8 y_R, 9 combine y = y_L + y_R, 10 end.
    Edges: start to every vertex without another predecessor; Pack ->
    PostSends; PostSends -> WaitSend; PostRecvs -> WaitRecv; WaitRecv -> y_R;
    y_L -> combine; y_R -> combine; WaitSend -> end; combine -> end.
    Returns (vertices, edges, kind) with kind[v] in {"CPU", "GPU"}.
    """
    v = list(range(1, 11))
    edges = [(1, 2), (1, 3), (1, 5), (2, 4), (4, 6), (5, 7), (7, 8),
             (3, 9), (8, 9), (6, 10), (9, 10)]
    kind = {1: "CPU", 2: "GPU", 3: "GPU", 4: "CPU", 5: "CPU", 6: "CPU",
            7: "CPU", 8: "GPU", 9: "GPU", 10: "CPU"}
    return v, edges, kind


# ------------------------------------------------------------------ #
# Traversals                                                          #
# ------------------------------------------------------------------ #
def is_topological(order, edges):
    """True when ``order`` lists every vertex once and each edge u -> v has
    u before v (Sec. III-B: all dependencies of a vertex complete first)."""
    pos = {}
    for i, v in enumerate(order):
        if v in pos:
            return False
        pos[v] = i
    for u, v in edges:
        if u not in pos or v not in pos or pos[u] >= pos[v]:
            return False
    return True


def is_canonical_streams(order, stream_of, gpu_ops):
    """Streams numbered by first use along the order (bijection pruning)."""
    nxt = 0
    for v in order:
        if v not in gpu_ops:
            continue
        s = stream_of[v]
        if s > nxt or s < 0:
            return False
        if s == nxt:
            nxt += 1
    return True


def brute_force_schedules(ops, edges, n_streams, gpu_ops=None):
    """Every (order, stream map) pair, by filtering all permutations of the
    ops times all maps of the GPU ops to streams.  Returns a list of
    (order tuple, stream tuple indexed by op id, -1 for CPU ops)."""
    gpu_ops = set(ops) if gpu_ops is None else set(gpu_ops)
    gpu_list = [v for v in ops if v in gpu_ops]
    size = max(ops) + 1
    out = []
    for order in itertools.permutations(ops):
        if not is_topological(order, edges):
            continue
        for assign in itertools.product(range(n_streams), repeat=len(gpu_list)):
            stream_of = [-1] * size
            for v, s in zip(gpu_list, assign):
                stream_of[v] = s
            if is_canonical_streams(order, stream_of, gpu_ops):
                out.append((tuple(order), tuple(stream_of)))
    return out


def count_brute_force(ops, edges, n_streams, gpu_ops=None):
    return len(brute_force_schedules(ops, edges, n_streams, gpu_ops))


# ------------------------------------------------------------------ #
# Table III                                                            #
# ------------------------------------------------------------------ #
def sync_for_edge(u_type, u_stream, v_type, v_stream):
    """The synchronisation Table III inserts for a DAG edge u -> v.

    Types are "CPU" or "GPU" (a BoundGPU vertex with its stream).  Returns a
    list of CUDA calls, empty when none is needed.
    """
    if u_type == "CPU":
        return []                                   # CPU ops are synchronous
    if v_type == "CPU":
        return ["cudaEventRecord", "cudaEventSynchronize"]
    if u_stream == v_stream:
        return []                                   # same stream: in order
    return ["cudaEventRecord", "cudaStreamWaitEvent"]


def sync_counts(edges, stream_of, kinds=None):
    """Records and waits of one implementation under Table III, with a
    record placed right after its producer and shared by all of the
    producer's cross-stream successors, and one wait per cross-stream edge.
    ``kinds`` maps a vertex to "CPU"/"GPU" (default: all GPU).
    Returns (records, stream_waits, event_syncs)."""
    recorded = set()
    waits = syncs = 0
    for u, v in edges:
        ku = kinds[u] if kinds else "GPU"
        kv = kinds[v] if kinds else "GPU"
        calls = sync_for_edge(ku, stream_of[u] if ku == "GPU" else None,
                              kv, stream_of[v] if kv == "GPU" else None)
        if "cudaEventRecord" in calls:
            recorded.add(u)
        waits += calls.count("cudaStreamWaitEvent")
        syncs += calls.count("cudaEventSynchronize")
    return len(recorded), waits, syncs


def sync_op_names(order, stream_of, edges, names, kinds=None):
    """The traversal with Table III's operations inserted and named after
    the paper's convention ("CER-after-Pack", "CES-b4-PostSend"): a record
    right after its producer, a wait or synchronize right before its
    consumer.  Returns the list of names."""
    succ = {}
    pred = {}
    for u, v in edges:
        succ.setdefault(u, []).append(v)
        pred.setdefault(v, []).append(u)
    kinds = kinds or {v: "GPU" for v in order}
    out = []
    for v in order:
        for u in pred.get(v, []):
            calls = sync_for_edge(kinds[u], stream_of[u], kinds[v], stream_of[v])
            if "cudaEventSynchronize" in calls:
                out.append("CES-b4-%s" % names[v])
            if "cudaStreamWaitEvent" in calls:
                out.append("CSWE-%s-b4-%s" % (names[u], names[v]))
        out.append(names[v])
        needs = any("cudaEventRecord" in sync_for_edge(kinds[v], stream_of[v],
                                                        kinds[w], stream_of[w])
                    for w in succ.get(v, []))
        if needs:
            out.append("CER-after-%s" % names[v])
    return out
