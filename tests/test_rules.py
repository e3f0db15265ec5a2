"""Design-rule stage (Sec. IV): labels, features, Alg. 1 tree and rule text,
on planted data where the answer is known."""
import numpy as np
import pytest

from oracle import schedules as OS
from paper_2203_02530_gb300 import rules as R
from paper_2203_02530_gb300 import schedules as E

pytest.importorskip("scipy")


def test_step_convolution_matches_definition():
    rng = np.random.default_rng(0)
    a = np.sort(rng.random(40))
    for r in (1, 2, 5):
        c, base = R.step_convolution(a, r)
        assert base == r - 1
        for j, i in enumerate(range(r - 1, 40 - r)):
            want = sum(a[i + m] for m in range(1, r + 1)) - sum(a[i + m] for m in range(-r + 1, 1))
            assert c[j] == pytest.approx(want)


def test_class_labels_on_three_levels():
    # equal steps without noise: exactly the two steps are class boundaries
    rng = np.random.default_rng(1)
    t = np.concatenate([np.full(500, 1.0), np.full(300, 2.0), np.full(200, 3.0)])
    perm = rng.permutation(t.size)
    lab, bounds = R.class_labels(t[perm])
    assert bounds == [499, 799]
    back = np.empty_like(lab)
    back[perm] = lab
    assert (back[:500] == 0).all() and (back[500:800] == 1).all() and (back[800:] == 2).all()


def test_class_labels_keep_the_true_steps_among_noise_peaks():
    # with noise the 98th-percentile cut keeps the top 2 % of all peaks,
    # which must include both steps
    rng = np.random.default_rng(1)
    t = np.sort(np.concatenate([1.0 + 0.01 * rng.random(500), 2.0 + 0.01 * rng.random(300),
                                3.0 + 0.01 * rng.random(200)]))
    lab, bounds = R.class_labels(t)
    assert 499 in bounds and 799 in bounds
    assert lab[0] == 0 and lab[-1] == len(bounds)


def test_expand_inserts_table3_operations():
    ops, edges = OS.coarse_dag()
    names = R.coarse_names()
    # pack, copy on stream 0; local, remote on stream 1
    seq = R.expand([0, 1, 2, 3], [0, 1, 0, 1], edges, names)
    assert seq == ["Pack", "yL", "Copy", "CER-after-Copy", "CSW-Copy-b4-yR", "yR"]
    # everything on one stream: nothing inserted
    assert R.expand([0, 1, 2, 3], [0, 0, 0, 0], edges, names) == names


def _planted_records():
    ops, edges = OS.coarse_dag()
    names = R.coarse_names()
    recs = []
    rng = np.random.default_rng(2)
    for o, s in E.enumerate_schedules(E.Dag(4, edges), 2):
        fast = o.index(0) < o.index(1) and s[0] != s[1]    # Pack before yL, other stream
        recs.append((o, s, (1.0 if fast else 2.0) + 1e-3 * rng.random()))
    return recs, edges, names


def test_tree_recovers_a_planted_rule():
    pytest.importorskip("sklearn")
    recs, edges, names = _planted_records()
    t = np.array([r[2] for r in recs])
    lab, _ = R.class_labels(t)
    assert set(lab.tolist()) == {0, 1}
    X, cols = R.feature_matrix(recs, edges, names)
    clf, mln, hist = R.search_tree(X, lab)
    assert clf.score(X, lab) == 1.0
    sets = R.rulesets(clf, cols)
    text = " ".join(" ".join(rs) for _, rs in sets[0])
    assert "Pack before yL" in text
    assert "Pack, yL different streams" in text
    # Alg. 1 only accepts a larger tree when its error is lower
    accepted = [h[1] for h in hist]
    assert min(accepted) == accepted[-1] or accepted[-1] >= min(accepted)


def test_accuracy_protocol_is_one_on_the_full_set():
    pytest.importorskip("sklearn")
    recs, edges, names = _planted_records()
    acc = R.accuracy_vs_iterations(recs, edges, names, [len(recs)])
    assert acc[0][1] == 1.0


def test_report_renders():
    pytest.importorskip("sklearn")
    recs, edges, names = _planted_records()
    text = R.report(recs, edges, names, "planted")
    assert "Class 0" in text and "class accuracy" in text


def test_method_constants_come_from_one_place():
    """The search, the measurement protocol and the rule stage read the
    paper's constants from one frozen dataclass: c = sqrt(2) (Sec. III-C.1),
    0.01 s per measurement (Sec. III-C.3), radius 0.5 % and the 98th
    percentile (Sec. IV-A), gini with balanced weights (Table IV), Alg. 1
    starting at 2 leaves and trying 5 more."""
    import dataclasses
    import inspect
    import math
    from paper_2203_02530_gb300 import benchmark, mcts, rules
    from paper_2203_02530_gb300.constants import PAPER
    assert PAPER.c_explore == math.sqrt(2.0) and mcts.C_EXPLORE == PAPER.c_explore
    assert PAPER.t_measure == 0.01 and benchmark.T_MEASURE == PAPER.t_measure
    sig = inspect.signature(rules.class_labels)
    assert sig.parameters["radius_frac"].default == PAPER.label_radius_frac == 0.005
    assert sig.parameters["percentile"].default == PAPER.prominence_percentile == 98.0
    assert (PAPER.tree_criterion, PAPER.tree_class_weight) == ("gini", "balanced")
    assert (PAPER.tree_first_leaves, PAPER.tree_more_leaves) == (2, 5)
    with pytest.raises(dataclasses.FrozenInstanceError):
        PAPER.t_measure = 1.0
