"""Closed forms of the paper's worst-case reachability results (Table 1).

These are used only as pins: a pruned graph built by the oracle must have a
measured reachability at least as large as the worst case the paper proves.
"""
import math


def unsorted_bound(a1: float, a2: float) -> float:
    """Theorem 3.1 (any metric, unsorted), as its proof derives it:
    a1 a2 / (a1 + a2 + 1), i.e. 1 / (1/a1 + 1/a2 + 1/(a1 a2)).

    Table 1 and the statement of Theorem 3.1 print 1 / (1/a1 + 1/a2 + 1); the
    proof (upper bound via the triangle inequality, attained by the collinear
    points of Lemma 3.5) gives the value above, which the construction attains.
    """
    return a1 * a2 / (a1 + a2 + 1.0)


def unsorted_bound_as_printed(a1: float, a2: float) -> float:
    """Table 1 / Theorem 3.1 as printed: 1 / (1/a1 + 1/a2 + 1) (never larger than
    :func:`unsorted_bound`, so it remains a valid, weaker lower bound)."""
    return 1.0 / (1.0 / a1 + 1.0 / a2 + 1.0)


def sorted_general_bound(a1: float, a2: float) -> float:
    """Theorem 3.2, first item (any metric, sorted): 1 / (1/a1 + 1/a2)."""
    return 1.0 / (1.0 / a1 + 1.0 / a2)


def beta_euc(a1: float, a2: float) -> float:
    """Lemma 3.8: (1/a1) sqrt(1 - 1/(4 a2^2)) + (1/a2) sqrt(1 - 1/(4 a1^2))."""
    return (1.0 / a1) * math.sqrt(1.0 - 1.0 / (4.0 * a2 * a2)) + \
        (1.0 / a2) * math.sqrt(1.0 - 1.0 / (4.0 * a1 * a1))


def sorted_euclid_bound(a1: float, a2: float) -> float:
    """Theorem 3.2, second item (Euclidean, sorted): 1 / beta_euc(a1, a2)."""
    return 1.0 / beta_euc(a1, a2)


def appendix_a_points(a1: float, a2: float):
    """Appendix A lower-bound construction: z=(1,0), y at angle 2*t1, x at angle
    2*(t1+t2) on the unit circle around p=(0,0), t_i = asin(1/(2 a_i))."""
    t1 = math.asin(1.0 / (2.0 * a1))
    t2 = math.asin(1.0 / (2.0 * a2))
    p = (0.0, 0.0)
    z = (1.0, 0.0)
    y = (math.cos(2 * t1), math.sin(2 * t1))
    x = (math.cos(2 * (t1 + t2)), math.sin(2 * (t1 + t2)))
    return p, x, y, z
