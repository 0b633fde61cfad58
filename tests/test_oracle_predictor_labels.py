"""The predictor's soft labels: the cheapest grid point dominates, ties share."""
import math

import numpy as np

import __graft_entry__

__graft_entry__._build_module().build()          # the package loads libfd.so on import
from paper_2209_01974_gb300 import predictor as pr  # noqa: E402


def _cost(best_i, best_j, others=2.0):
    c = np.full((1, len(pr.GRID_CN), len(pr.GRID_M)), others)
    c[0, best_i, best_j] = 1.0
    return c


def test_soft_label_picks_a_clear_minimum():
    lab = pr.soft_labels(_cost(2, 0))[0]
    assert abs(lab[0] - math.log(pr.GRID_CN[2])) < 1e-6 and abs(lab[1] - pr.GRID_M[0]) < 1e-6


def test_soft_label_averages_ties_and_skips_failures():
    shape = (1, len(pr.GRID_CN), len(pr.GRID_M))
    c = np.full(shape, np.inf)
    c[0, 0, 0] = c[0, 2, 2] = 100.0
    lab = pr.soft_labels(c)[0]
    assert abs(lab[0] - 0.5 * (math.log(pr.GRID_CN[0]) + math.log(pr.GRID_CN[2]))) < 1e-6
    assert abs(lab[1] - 0.5 * (pr.GRID_M[0] + pr.GRID_M[2])) < 1e-6
    lab = pr.soft_labels(np.full(shape, np.inf))[0]
    assert abs(lab[0] - math.log(4.0)) < 1e-6 and lab[1] == 0.5
