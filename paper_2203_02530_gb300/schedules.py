"""Implementations of an operation DAG: topological orders with a stream
binding per operation (Sec. III-B, Eq. 1; Table II BoundGPU vertices),
pruned of stream relabellings (Sec. III-C.2).

Canonical form: streams are numbered by first use along the order, so the
first operation is on stream 0 and every operation uses a stream already in
use or the next unused number.  The enumerator walks prefixes P_k depth
first (the sequential-decision view of Sec. III-B), extending a prefix by
every ready operation on every admissible stream.
"""
import math
from functools import lru_cache


class Dag:
    """Operations 0..n_ops-1 and dependency edges (u, v): u before v."""

    def __init__(self, n_ops, edges):
        self.n_ops = int(n_ops)
        self.edges = [(int(u), int(v)) for u, v in edges]
        self.pred_mask = [0] * self.n_ops
        for u, v in self.edges:
            self.pred_mask[v] |= 1 << u

    def ready(self, done_mask):
        """Operations not yet issued whose predecessors all are."""
        return [v for v in range(self.n_ops)
                if not done_mask >> v & 1 and self.pred_mask[v] & done_mask == self.pred_mask[v]]

    def is_topological(self, order):
        done = 0
        if sorted(order) != list(range(self.n_ops)):
            return False
        for v in order:
            if self.pred_mask[v] & done != self.pred_mask[v]:
                return False
            done |= 1 << v
        return True


def coarse_spmv_dag():
    """pack -> copy -> remote, local -> remote (op ids 0..3 = pack, local,
    copy, remote)."""
    return Dag(4, [(0, 2), (2, 3), (1, 3)])


def children(dag, done_mask, n_used, n_streams):
    """Legal next decisions (op, stream) from a prefix: every ready op on a
    stream already used or the next unused one."""
    out = []
    for v in dag.ready(done_mask):
        for s in range(min(n_used + 1, n_streams)):
            out.append((v, s))
    return out


def enumerate_schedules(dag, n_streams, limit=None):
    """Yield (order, stream_of_op) for every canonical implementation."""
    order, smap = [], [0] * dag.n_ops
    count = [0]

    def rec(done, n_used):
        if limit is not None and count[0] >= limit:
            return
        if len(order) == dag.n_ops:
            count[0] += 1
            yield list(order), list(smap)
            return
        for v, s in children(dag, done, n_used, n_streams):
            order.append(v)
            smap[v] = s
            yield from rec(done | 1 << v, max(n_used, s + 1))
            order.pop()

    yield from rec(0, 0)


def count_schedules(dag, n_streams):
    """Number of canonical implementations, by dynamic programming over
    (issued set, streams in use)."""

    @lru_cache(maxsize=None)
    def f(done, n_used):
        if done == (1 << dag.n_ops) - 1:
            return 1
        return sum(f(done | 1 << v, max(n_used, s + 1))
                   for v, s in children(dag, done, n_used, n_streams))

    return f(0, 0)


def canonicalize(order, stream_of_op):
    """Relabel streams by first use along the order."""
    remap, out = {}, list(stream_of_op)
    for v in order:
        s = stream_of_op[v]
        if s not in remap:
            remap[s] = len(remap)
        out[v] = remap[s]
    return out


def stirling2(m, k):
    return sum((-1) ** j * math.comb(k, j) * (k - j) ** m for j in range(k + 1)) // math.factorial(k)


def stream_map_counts(n_ops, n_streams):
    """g[r][k]: canonical stream bindings of r more operations when k streams
    are already in use.  Each operation takes one of the k streams in use or,
    while k < n_streams, opens the next one; the count does not depend on
    which operations these are or in what order they come:
    g[0][k] = 1, g[r][k] = k g[r-1][k] + [k < S] g[r-1][k+1]."""
    S = int(n_streams)
    g = [[1] * (S + 1)]
    for r in range(1, n_ops + 1):
        prev = g[-1]
        g.append([k * prev[k] + (prev[k + 1] if k < S else 0) for k in range(S + 1)])
    return g


class UniformSampler:
    """Draws canonical implementations uniformly over all of them (the
    random-sampling baseline of Sec. VI, against which MCTS is compared).

    The implementations reachable from a prefix number e(done) * g[r][k]:
    e(done) is the count of topological orders of the operations not yet
    issued (a dynamic program over the DAG's downsets, memoised), g the
    stream bindings above (r operations left, k streams in use).  Each step
    takes ready operation v with probability e(done | v) / e(done) and then
    a stream in use with probability g[r-1][k] / g[r][k] each, or the next
    stream with probability g[r-1][k+1] / g[r][k]; the product of the
    step probabilities is 1 / (e(0) g[n][0]) for every implementation."""

    def __init__(self, dag, n_streams, max_states=5_000_000):
        self.dag = dag
        self.S = int(n_streams)
        self.full = (1 << dag.n_ops) - 1
        self.g = stream_map_counts(dag.n_ops, self.S)
        self.max_states = max_states
        self._e = {self.full: 1}
        self._count_orders()

    def _count_orders(self):
        # downsets reached from the empty prefix, then e() from the full
        # set back (iterative: no recursion limit, one pass per downset)
        dag, seen, stack, topo = self.dag, {0}, [0], []
        while stack:
            d = stack.pop()
            topo.append(d)
            for v in dag.ready(d):
                nd = d | 1 << v
                if nd not in seen:
                    if len(seen) >= self.max_states:
                        raise ValueError("more than %d downsets: the DAG is too wide to count" % self.max_states)
                    seen.add(nd)
                    stack.append(nd)
        for d in sorted(topo, key=lambda m: -bin(m).count("1")):
            if d != self.full:
                self._e[d] = sum(self._e[d | 1 << v] for v in dag.ready(d))
        self.n_downsets = len(seen)

    def orders(self, done=0):
        """Topological orders of the operations outside `done` (a downset)."""
        return self._e[done]

    def total(self):
        """Canonical implementations: orders x stream bindings."""
        return self._e[0] * self.g[self.dag.n_ops][0]

    def draw(self, rng):
        """One implementation (order, stream_of_op); rng: random.Random."""
        dag, g = self.dag, self.g
        done, used, order, smap = 0, 0, [], [0] * dag.n_ops
        left = dag.n_ops
        while done != self.full:
            ready = dag.ready(done)
            u = rng.randrange(self._e[done])
            for v in ready:
                u -= self._e[done | 1 << v]
                if u < 0:
                    break
            w = rng.randrange(g[left][used])
            s = w // g[left - 1][used] if w < used * g[left - 1][used] else used
            order.append(v)
            smap[v] = s
            used = max(used, s + 1)
            done |= 1 << v
            left -= 1
        return order, smap


def draw_per_decision(dag, n_streams, rng):
    """One implementation completed by uniformly random legal decisions from
    the empty prefix (the rollout of Sec. III-C without a tree).  Not uniform
    over implementations: a decision leading to fewer completions is taken
    as often as one leading to many."""
    full = (1 << dag.n_ops) - 1
    done, used, order, smap = 0, 0, [], [0] * dag.n_ops
    while done != full:
        opts = children(dag, done, used, n_streams)
        v, s = opts[rng.randrange(len(opts))]
        order.append(v)
        smap[v] = s
        used = max(used, s + 1)
        done |= 1 << v
    return order, smap


def sample_programs(dag, n_streams, count, seed=0, mode="uniform", max_draws=None):
    """`count` distinct implementations drawn at random (all of them, in a
    random order, when the space holds no more than `count`).
    mode "uniform": every implementation equally likely (UniformSampler);
    "per_decision": uniformly random legal decisions (draw_per_decision)."""
    import random
    rng = random.Random(seed)
    if mode == "uniform":
        sampler = UniformSampler(dag, n_streams)
        total = sampler.total()
        draw = lambda: sampler.draw(rng)
    elif mode == "per_decision":
        total = count_schedules(dag, n_streams) if dag.n_ops <= 16 else None
        draw = lambda: draw_per_decision(dag, n_streams, rng)
    else:
        raise ValueError("mode %r" % (mode,))
    if total is not None and total <= count:
        out = [(o, m) for o, m in enumerate_schedules(dag, n_streams)]
        rng.shuffle(out)
        return out
    seen, out, draws = set(), [], 0
    limit = max_draws if max_draws is not None else 50 * count + 10_000
    while len(out) < count and draws < limit:
        draws += 1
        o, m = draw()
        key = (tuple(o), tuple(m))
        if key in seen:
            continue
        seen.add(key)
        out.append((o, m))
    return out
