"""Design-rule generation from measured implementations (Sec. IV).

Input: records (order, stream map, seconds) of implementations of an
operation DAG, e.g. from the MCTS search.  Steps:

  class labels (Sec. IV-A)  sort the times; convolve with a step kernel of
      radius r = max(1, floor(0.005 * count)) (-1 on the r samples up to
      and including i, +1 on the r samples after i), only where the kernel
      fits; keep the peaks whose prominence is at least the 98th percentile
      of all peak prominences (scipy.signal.find_peaks); a peak at i is a
      class boundary between sorted samples i and i + 1.
  features (Sec. IV-B)      expand each traversal with the synchronisation
      operations Table III inserts (an event record after an operation that
      feeds another stream, a stream wait before an operation fed from
      another stream); one ordering feature per pair of operations ("u
      before v"; 0 when either is absent), one stream feature per pair of
      GPU operations ("u, v same stream"); constant columns dropped.
  tree (Sec. IV-C, Table IV, Alg. 1)   CART with gini, balanced class
      weights, max_depth = max_leaf_nodes - 1; max_leaf_nodes grown from 2
      while the training error falls, trying +1 .. +5.
  rules (Sec. IV-D)         every root-to-leaf path is a ruleset for the
      leaf's class; rulesets are ordered by the samples they cover.
  accuracy (Sec. V, Table V)    labels, tree and class time ranges from the
      first N records classify every implementation; accuracy is the share
      whose time lies in its predicted class's range.

scikit-learn and scipy are needed for this stage only (host side).
"""
import json
import math

import numpy as np

from .constants import PAPER


# ---------------------------------------------------------------- labels
def step_convolution(a, r):
    """c[i] = sum(a[i+1 .. i+r]) - sum(a[i-r+1 .. i]) for r-1 <= i <= len-1-r.
    Returns (c, first index i of c)."""
    a = np.asarray(a, dtype=np.float64)
    n = a.size
    if n < 2 * r:
        return np.zeros(0), 0
    cs = np.concatenate([[0.0], np.cumsum(a)])
    i = np.arange(r - 1, n - r)
    after = cs[i + r + 1] - cs[i + 1]
    upto = cs[i + 1] - cs[i - r + 1]
    return after - upto, r - 1


def class_labels(times, radius_frac=PAPER.label_radius_frac, percentile=PAPER.prominence_percentile):
    """Class of every time (0 = fastest), in the input order, and the sorted
    positions after which a new class starts."""
    from scipy.signal import find_peaks
    t = np.asarray(times, dtype=np.float64)
    order = np.argsort(t, kind="stable")
    a = t[order]
    r = max(1, int(math.floor(radius_frac * a.size)))
    c, base = step_convolution(a, r)
    bounds = []
    if c.size >= 3:
        peaks, props = find_peaks(c, prominence=0.0)
        if peaks.size:
            prom = props["prominences"]
            thr = np.percentile(prom, percentile)
            bounds = sorted(int(p + base) for p, q in zip(peaks, prom) if q >= thr and q > 0)
    sorted_label = np.zeros(a.size, dtype=np.int64)
    for b in bounds:
        sorted_label[b + 1:] += 1
    labels = np.empty_like(sorted_label)
    labels[order] = sorted_label
    return labels, bounds


# ---------------------------------------------------------------- features
def expand(order, smap, edges, names, gpu_ops=None):
    """The traversal with Table III's operations inserted and named:
    'CER-after-<u>' right after an op that feeds an op on another stream,
    'CSW-<u>-b4-<v>' right before v for each such predecessor u."""
    gpu = set(range(len(smap))) if gpu_ops is None else set(gpu_ops)
    succ, pred = {}, {}
    for u, v in edges:
        succ.setdefault(u, []).append(v)
        pred.setdefault(v, []).append(u)
    out = []
    for v in order:
        for u in pred.get(v, []):
            if u in gpu and v in gpu and smap[u] != smap[v]:
                out.append("CSW-%s-b4-%s" % (names[u], names[v]))
        out.append(names[v])
        if v in gpu and any(w in gpu and smap[w] != smap[v] for w in succ.get(v, [])):
            out.append("CER-after-%s" % names[v])
    return out


def feature_matrix(records, edges, names, gpu_ops=None, columns=None):
    """Binary features of every record; returns (X, column names).  With
    `columns` given, exactly those features are built (for classifying new
    records with a trained tree)."""
    seqs = [expand(o, s, edges, names, gpu_ops) for o, s, _ in records]
    gpu = sorted(set(range(len(names))) if gpu_ops is None else set(gpu_ops))
    if columns is None:
        ops = sorted({x for q in seqs for x in q})
        cols = [("order", u, v) for i, u in enumerate(ops) for v in ops[i + 1:]]
        cols += [("stream", names[u], names[v]) for i, u in enumerate(gpu) for v in gpu[i + 1:]]
    else:
        cols = list(columns)
    name_to_op = {names[i]: i for i in range(len(names))}
    X = np.zeros((len(records), len(cols)), dtype=np.int8)
    for r, ((o, smap, _), q) in enumerate(zip(records, seqs)):
        pos = {x: i for i, x in enumerate(q)}
        for c, (kind, u, v) in enumerate(cols):
            if kind == "order":
                X[r, c] = 1 if (u in pos and v in pos and pos[u] < pos[v]) else 0
            else:
                X[r, c] = 1 if smap[name_to_op[u]] == smap[name_to_op[v]] else 0
    if columns is None:
        keep = [c for c in range(len(cols)) if X[:, c].min() != X[:, c].max()]
        X = X[:, keep]
        cols = [cols[c] for c in keep]
    return X, cols


def column_text(col, value):
    kind, u, v = col
    if kind == "order":
        return "%s before %s" % (u, v) if value else "%s before %s" % (v, u)
    return "%s, %s same stream" % (u, v) if value else "%s, %s different streams" % (u, v)


# ---------------------------------------------------------------- tree
def train(X, y, max_leaf_nodes, seed=0):
    """(training error, classifier) with the parameters of Table IV."""
    from sklearn.tree import DecisionTreeClassifier
    clf = DecisionTreeClassifier(criterion=PAPER.tree_criterion, max_leaf_nodes=max_leaf_nodes,
                                 max_depth=max(1, max_leaf_nodes - 1),
                                 class_weight=PAPER.tree_class_weight, random_state=seed)
    clf.fit(X, y)
    return 1.0 - clf.score(X, y), clf


def search_tree(X, y, seed=0):
    """Alg. 1: grow max_leaf_nodes from 2 while the training error falls,
    trying up to 5 more leaves each time.  Returns (clf, mln, history)."""
    mln = PAPER.tree_first_leaves
    err = math.inf
    cur, clf = train(X, y, mln, seed)
    history = [(mln, cur, clf.get_depth())]
    while cur < err:
        err = cur
        for i in range(1, PAPER.tree_more_leaves + 1):
            cur, nclf = train(X, y, mln + i, seed)
            history.append((mln + i, cur, nclf.get_depth()))
            if cur < err:
                clf = nclf
                mln = mln + i
                break
    return clf, mln, history


def rulesets(clf, columns):
    """{class: [(samples, [rule text, ...]), ...]} from root-to-leaf paths,
    each class's rulesets ordered by the samples they cover."""
    t = clf.tree_
    out = {}

    def walk(node, path):
        if t.children_left[node] == -1:
            cls = int(clf.classes_[int(np.argmax(t.value[node][0]))])
            out.setdefault(cls, []).append((int(t.n_node_samples[node]), list(path)))
            return
        col = columns[t.feature[node]]
        walk(t.children_left[node], path + [column_text(col, 0)])    # feature <= 0.5
        walk(t.children_right[node], path + [column_text(col, 1)])
    walk(0, [])
    for k in out:
        out[k].sort(key=lambda r: -r[0])
    return out


# ---------------------------------------------------------------- Table V
def class_ranges(times, labels):
    return {int(c): (float(np.min(times[labels == c])), float(np.max(times[labels == c])))
            for c in np.unique(labels)}


def accuracy_vs_iterations(records, edges, names, sizes, everything=None, gpu_ops=None, seed=0):
    """For each N in sizes: labels, features and a tree from the first N
    records (search order); classify every implementation of `everything`
    (default: all records) and report the share whose time lies in the
    predicted class's range."""
    everything = records if everything is None else everything
    t_all = np.array([r[2] for r in everything])
    out = []
    for n in sizes:
        sub = records[:n]
        t = np.array([r[2] for r in sub])
        lab, _ = class_labels(t)
        X, cols = feature_matrix(sub, edges, names, gpu_ops)
        if X.shape[1] == 0 or len(np.unique(lab)) < 2:
            pred = np.zeros(len(everything), dtype=np.int64)
            rng_ = class_ranges(t, lab)
        else:
            clf, _, _ = search_tree(X, lab, seed)
            Xa, _ = feature_matrix(everything, edges, names, gpu_ops, columns=cols)
            pred = clf.predict(Xa)
            rng_ = class_ranges(t, lab)
        ok = [rng_[int(p)][0] <= ta <= rng_[int(p)][1] for p, ta in zip(pred, t_all)]
        out.append((n, float(np.mean(ok)), int(len(np.unique(lab)))))
    return out


# ---------------------------------------------------------------- report
def coarse_names():
    return ["Pack", "yL", "Copy", "yR"]


def per_rank_names(P):
    return ["%s%d" % (k, p) for p in range(P) for k in ("Pack", "yL", "Copy", "yR")]


def load_records(path):
    recs = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line:
                r = json.loads(line)
                recs.append((r["order"], r["streams"], float(r["seconds"])))
    return recs


def report(records, edges, names, title, sizes=(50, 100, 200, 400)):
    """Markdown text: classes, the tree found by Alg. 1, three rulesets per
    class, and the Table V protocol on the records given."""
    t = np.array([r[2] for r in records])
    lab, bounds = class_labels(t)
    X, cols = feature_matrix(records, edges, names)
    lines = ["# %s" % title, "",
             "%d implementations; fastest %.2f us, slowest %.2f us (spread %.3fx)." % (
                 len(records), t.min() * 1e6, t.max() * 1e6, t.max() / t.min()), ""]
    rng_ = class_ranges(t, lab)
    lines.append("Classes (Sec. IV-A): " + ", ".join(
        "%d: %d programs, %.2f-%.2f us" % (c, int((lab == c).sum()), lo * 1e6, hi * 1e6)
        for c, (lo, hi) in sorted(rng_.items())))
    lines.append("")
    if X.shape[1] and len(np.unique(lab)) > 1:
        clf, mln, hist = search_tree(X, lab)
        lines.append("Alg. 1 settled on max_leaf_nodes = %d (depth %d, training error %.3f); "
                     "%d features after dropping constant ones." % (
                         mln, clf.get_depth(), 1.0 - clf.score(X, lab), X.shape[1]))
        lines.append("")
        for c, sets in sorted(rulesets(clf, cols).items()):
            lines.append("## Class %d" % c)
            for n_s, rs in sets[:3]:
                lines.append("- (%d samples) " % n_s + "; ".join(rs))
            lines.append("")
    sizes = [s for s in sizes if s < len(records)] + [len(records)]
    acc = accuracy_vs_iterations(records, edges, names, sizes)
    lines.append("| records used | " + " | ".join(str(a[0]) for a in acc) + " |")
    lines.append("|---" * (len(acc) + 1) + "|")
    lines.append("| class accuracy | " + " | ".join("%.2f" % a[1] for a in acc) + " |")
    lines.append("")
    return "\n".join(lines)


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="design rules from a JSONL record log")
    ap.add_argument("records")
    ap.add_argument("--dag", required=True, help="JSON file with n_ops, edges and optional P")
    ap.add_argument("--title", default="Design rules")
    a = ap.parse_args()
    d = json.load(open(a.dag))
    if "names" in d:
        names = d["names"]
    else:
        names = coarse_names() if d["n_ops"] == 4 else per_rank_names(d["n_ops"] // 4)
    print(report(load_records(a.records), [tuple(e) for e in d["edges"]], names, a.title))
