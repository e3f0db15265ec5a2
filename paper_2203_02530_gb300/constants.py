"""The method's constants in one place, each with the passage that fixes it.

Host-side only: the search (MCTS), the measurement protocol and the design-rule
stage read them from here; kernel tunables live in the autotuner's cache.
"""
import math
from dataclasses import dataclass


@dataclass(frozen=True)
class PaperConstants:
    # MCTS child selection: c * sqrt(ln N / n) + V (Sec. III-C.1)
    c_explore: float = math.sqrt(2.0)
    # a measurement repeats samples until this many seconds have elapsed (Sec. III-C.3)
    t_measure: float = 0.01
    # class labels: step-kernel radius as a fraction of the sample count, at least 1,
    # and the prominence percentile a peak must reach (Sec. IV-A)
    label_radius_frac: float = 0.005
    prominence_percentile: float = 98.0
    # decision tree (Table IV): split criterion and class weighting
    tree_criterion: str = "gini"
    tree_class_weight: str = "balanced"
    # Alg. 1: the first max_leaf_nodes, and how many larger sizes each step tries
    tree_first_leaves: int = 2
    tree_more_leaves: int = 5


PAPER = PaperConstants()
