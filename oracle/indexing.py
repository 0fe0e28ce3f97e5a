"""Index sets and linearisation functions of Sec. 4 (oracle, test infrastructure).

* ``n_tet``/``n_tri``: cardinalities of I_tet(w), I_tri(w) (Sec. 3.2, Eqs.
  for the tetrahedral and triangular numbers).
* ``tw``: the map t_w(i,j,k) (Sec. 4, linearisation equation), closed form.
* ``tw_by_counting``: the same map obtained by numbering I_tet(w) in the loop
  order the paper gives for consecutive access (k outermost, then j, i
  innermost).  The two must agree; pinned in tests.
* ``aos``/``soa``: layouts for m scalars per micro-primitive (Sec. 4).
* ``subgroup_widths``: Table 1, with the xyz-down micro-face width read as
  2^l - 1 (the table prints 2^l - 2; brute-force counting and the Euler
  characteristic both fix 2^l - 1).
"""
from __future__ import annotations


def n_tet(w: int) -> int:
    """w-th tetrahedral number |I_tet(w)| = w(w+1)(w+2)/6 (0 for w <= 0)."""
    return w * (w + 1) * (w + 2) // 6 if w > 0 else 0


def n_tri(w: int) -> int:
    """w-th triangular number |I_tri(w)| = w(w+1)/2 (0 for w <= 0)."""
    return w * (w + 1) // 2 if w > 0 else 0


def tw(w: int, i: int, j: int, k: int) -> int:
    """t_w(i,j,k) = N_tet(w) - N_tet(w-k) + N_tri(w-k) - N_tri(w-k-j) + i."""
    return n_tet(w) - n_tet(w - k) + n_tri(w - k) - n_tri(w - k - j) + i


def index_set_tet(w: int):
    """I_tet(w) = {(i,j,k) : i+j+k < w} as a list in the consecutive loop order."""
    return [(i, j, k) for k in range(w) for j in range(w - k) for i in range(w - k - j)]


def tw_by_counting(w: int) -> dict:
    """Number I_tet(w) 0,1,2,... in the order k outer, j middle, i inner."""
    return {p: n for n, p in enumerate(index_set_tet(w))}


def aos(w: int, m: int, i: int, j: int, k: int, d: int) -> int:
    """Array-of-structures index m * t_w(i,j,k) + d."""
    return m * tw(w, i, j, k) + d


def soa(w: int, m: int, i: int, j: int, k: int, d: int) -> int:
    """Structure-of-arrays index d * N_tet(w) + t_w(i,j,k)."""
    return d * n_tet(w) + tw(w, i, j, k)


def subgroup_widths(level: int) -> dict:
    """Table 1 side lengths w(l) of every micro-primitive subgroup."""
    n = 2 ** level
    return {
        ("vertex", "-"): n + 1,
        ("edge", "x"): n, ("edge", "y"): n, ("edge", "z"): n,
        ("edge", "xy"): n, ("edge", "xz"): n, ("edge", "yz"): n,
        ("edge", "xyz"): n - 1,
        ("face", "z-up"): n, ("face", "z-down"): n - 1,
        ("face", "y-up"): n, ("face", "y-down"): n - 1,
        ("face", "x-up"): n, ("face", "x-down"): n - 1,
        ("face", "xyz-up"): n, ("face", "xyz-down"): n - 1,  # table prints n-2
        ("face", "xy-up"): n - 1, ("face", "xy-down"): n - 1,
        ("face", "yz-up"): n - 1, ("face", "yz-down"): n - 1,
        ("cell", "I-up"): n, ("cell", "I-down"): n - 2,
        ("cell", "II-up"): n - 1, ("cell", "II-down"): n - 1,
        ("cell", "III-up"): n - 1, ("cell", "III-down"): n - 1,
    }
