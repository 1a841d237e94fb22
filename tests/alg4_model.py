"""Sequential model of Algorithm 4 (modified Apetrei with skips) for tests.

Each leaf "thread" of Algorithm 4 is a Python generator that yields right
before each atomic compare-and-swap on the ``store`` array, so a scheduler can
interleave the threads in any order. The model exists to test the paper's
algorithm as read (including the reading of its garbled left-child line)
against the top-down oracle under many arrival orders. It is test code only:
neither the oracle nor the CUDA library uses it.

delta* is computed from Python integers (keys augmented with their sorted
position, Sec. 3.2), +inf at -1 and n-1 (Sec. 3.1).

``left_child_rule``:
  * ``"split"`` - the reading used by the library: the parent's left child
    covers [range_left, p] where p is the split (the Apetrei index), so it is
    L_p when range_left == p and I_p otherwise (Sec. 4 text: the children of
    split gamma are gamma and gamma + 1).
  * ``"literal"`` - the line as printed in Algorithm 4 (compare range_left with
    q and name node i), kept to show that it does not reproduce Fig. 1.
"""
from __future__ import annotations

import random

INF = float("inf")
EMPTY = None  # the diamond value of Algorithm 4


def _dstar(sorted_codes):
    aug = [(int(c) << 32) | i for i, c in enumerate(sorted_codes)]
    n = len(aug)

    def d(i):
        if i < 0 or i >= n - 1:
            return INF
        return (aug[i] ^ aug[i + 1]).bit_length() - 1

    return d


def run(sorted_codes, seed=0, left_child_rule="split", schedule="random"):
    """Return dict(left, skip_internal, skip_leaf) in canonical ids."""
    n = len(sorted_codes)
    ni = n - 1
    d = _dstar(sorted_codes)
    left = [None] * max(ni, 0)
    skip_i = [None] * max(ni, 0)
    skip_l = [None] * n
    store = [EMPTY] * max(ni, 0)

    def L(k):
        return ni + k

    def I(k):
        return k

    def thread(i):
        range_left, delta_left = i, d(i - 1)
        range_right, delta_right = i, d(i)
        if i == n - 1:
            skip_l[i] = -1
        else:
            skip_l[i] = L(i + 1) if delta_right < d(i + 1) else I(i + 1)
        if n == 1:
            return
        while True:
            if delta_right < delta_left:  # left child of its parent
                p = range_right
                yield
                old = store[p]
                if old is EMPTY:
                    store[p] = range_left
                    return
                range_right = old
                delta_right = d(range_right)
            else:  # right child of its parent
                p = range_left - 1
                yield
                old = store[p]
                if old is EMPTY:
                    store[p] = range_right
                    return
                range_left = old
                delta_left = d(range_left - 1)
            q = range_right if delta_right < delta_left else range_left
            if left_child_rule == "split":
                left[q] = L(p) if range_left == p else I(p)
            else:
                left[q] = L(i) if range_left == q else I(i)
            if range_right == n - 1:
                skip_i[q] = -1
            else:
                r = range_right + 1
                skip_i[q] = L(r) if delta_right < d(r) else I(r)
            i = q
            if i == 0:
                return

    rng = random.Random(seed)
    live = [thread(i) for i in range(n)]
    if schedule == "reverse":
        live.reverse()
    while live:
        k = rng.randrange(len(live)) if schedule == "random" else 0
        try:
            next(live[k])
        except StopIteration:
            live.pop(k)
    return {"left": left, "skip_internal": skip_i, "skip_leaf": skip_l}
