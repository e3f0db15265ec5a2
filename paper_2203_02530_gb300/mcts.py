"""Monte-Carlo tree search over implementations of an operation DAG
(Sec. III-C).

A tree node is a prefix P_k of the program: the decisions (operation, stream)
taken so far.  Children are the legal next decisions: every ready operation
on every admissible stream, with streams numbered by first use so that
programs equal up to a stream relabelling are one program (Sec. III-C.2).

Each iteration:
  selection   from the root, descend to the child with the largest
              c * sqrt(ln N / n) + V, where N and n count the rollouts through
              the node and the child, c = sqrt(2), and
              V = (t_max^child - t_min^child) / (t_max^node - t_min^node)
              when n >= 2 and N >= 2, else 1; a fully explored child scores
              -inf; stop at a node that still has a child with no rollouts;
  expansion   create one such zero-rollout child (chosen uniformly);
  rollout     complete the program with random decisions, create the nodes
              on the way, and measure the program;
  backprop    update n, t_min and t_max of every node on the path.

Readings where the paper leaves a choice open: the random completion only
takes children whose subtrees are not fully explored, so no program is
measured twice and the search ends once every program has been measured;
ties in selection go to the first child in decision order.
"""
import math
import random

from .constants import PAPER
from .schedules import children

C_EXPLORE = PAPER.c_explore


class Node:
    __slots__ = ("parent", "decision", "done", "n_used", "kids", "legal", "n", "tmin", "tmax",
                 "explored")

    def __init__(self, parent, decision, done, n_used, legal):
        self.parent = parent
        self.decision = decision          # (op, stream) that led here
        self.done = done                  # bit mask of issued ops
        self.n_used = n_used              # streams in use
        self.kids = {}                    # decision -> Node
        self.legal = legal                # legal decisions from here
        self.n = 0                        # rollouts through this node
        self.tmin = math.inf
        self.tmax = -math.inf
        self.explored = False             # every program below measured


def exploit_value(child, parent):
    """V of Sec. III-C.1: the share of the parent's observed time range
    covered by the child's; 1 without two observations on either side."""
    if child.n >= 2 and parent.n >= 2:
        span = parent.tmax - parent.tmin
        if span <= 0.0:
            return 1.0
        return (child.tmax - child.tmin) / span
    return 1.0


class Mcts:
    """Search of `dag` (schedules.Dag) bound to `n_streams` streams.

    `evaluate(order, stream_of_op) -> seconds` measures one program.
    """

    def __init__(self, dag, n_streams, evaluate, seed=0, c=C_EXPLORE):
        self.dag = dag
        self.S = int(n_streams)
        self.evaluate = evaluate
        self.rng = random.Random(seed)
        self.c = c
        self.full = (1 << dag.n_ops) - 1
        self.root = self._node(None, None, 0, 0)
        self.records = []                 # (order, stream_of_op, seconds)

    def _node(self, parent, decision, done, n_used):
        legal = children(self.dag, done, n_used, self.S) if done != self.full else []
        return Node(parent, decision, done, n_used, legal)

    def _child(self, node, decision):
        ch = node.kids.get(decision)
        if ch is None:
            op, s = decision
            ch = self._node(node, decision, node.done | 1 << op, max(node.n_used, s + 1))
            node.kids[decision] = ch
        return ch

    @property
    def finished(self):
        return self.root.explored

    def _score(self, child, node):
        if child.explored:
            return -math.inf
        explore = self.c * math.sqrt(math.log(node.n) / child.n) if node.n > 0 and child.n > 0 else math.inf
        return explore + exploit_value(child, node)

    def _select(self):
        node = self.root
        while True:
            if node.done == self.full:
                return node
            if any(d not in node.kids or node.kids[d].n == 0 for d in node.legal):
                return node
            best, best_s = None, -math.inf
            for d in node.legal:
                sc = self._score(node.kids[d], node)
                if sc > best_s:
                    best, best_s = node.kids[d], sc
            if best is None:          # every child fully explored
                return node
            node = best

    def _expand(self, node):
        fresh = [d for d in node.legal
                 if (d not in node.kids or node.kids[d].n == 0) and
                 not (d in node.kids and node.kids[d].explored)]
        if not fresh:
            return node
        return self._child(node, fresh[self.rng.randrange(len(fresh))])

    def _rollout_path(self, node):
        path = []
        while node.done != self.full:
            opts = [d for d in node.legal if not (d in node.kids and node.kids[d].explored)]
            node = self._child(node, opts[self.rng.randrange(len(opts))])
            path.append(node)
        return node, path

    def _mark_explored(self, node):
        while node is not None:
            if node.done == self.full:
                node.explored = True
            elif len(node.kids) == len(node.legal) and all(k.explored for k in node.kids.values()):
                node.explored = True
            else:
                return
            node = node.parent

    def iterate(self):
        """One select / expand / rollout / backprop; returns the record, or
        None once every program has been measured."""
        if self.root.explored:
            return None
        leaf = self._expand(self._select())
        leaf, _ = self._rollout_path(leaf)
        order, smap = [], [0] * self.dag.n_ops
        node = leaf
        while node.parent is not None:
            op, s = node.decision
            order.append(op)
            smap[op] = s
            node = node.parent
        order.reverse()
        t = float(self.evaluate(order, smap))
        node = leaf
        while node is not None:
            node.n += 1
            node.tmin = min(node.tmin, t)
            node.tmax = max(node.tmax, t)
            node = node.parent
        self._mark_explored(leaf)
        rec = (order, smap, t)
        self.records.append(rec)
        return rec

    def run(self, iterations):
        for _ in range(int(iterations)):
            if self.iterate() is None:
                break
        return self.records

    def exploit_values(self):
        """Every (child, parent) V in the tree (for invariant checks)."""
        out, stack = [], [self.root]
        while stack:
            node = stack.pop()
            for ch in node.kids.values():
                out.append(exploit_value(ch, node))
                stack.append(ch)
        return out
