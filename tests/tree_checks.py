"""Independent checks of a linear BVH with skip connections.

These are written from the paper's statements, not from either
implementation, and are used to pin the oracle (and, in the GPU tests, to give
the CUDA tree a second, independent check):

* ``radix_tree_bruteforce`` - the binary radix tree of Sec. 3.1 by recursion
  over Python integers: a range of augmented keys splits where its highest
  differing bit flips.
* ``check_karras_tree`` - Sec. 3.1 invariants: n-1 internal nodes, each id used
  once, node i's range starts or ends at i, the root I_0 spans all keys, a left
  child is numbered by its range end and a right child by its range start, the
  index is the range bound with the smaller delta*, and the split is the unique
  argmax of delta* over the range.
* ``check_skips`` - Sec. 2 and Fig. 1: an always-true stackless walk (Algorithm
  1) visits all 2n-1 nodes in pre-order and reports leaves 0..n-1 once each, and
  every skip is the pre-order successor past the node's subtree; also Algorithm
  2's closed form for the skip target.
* ``check_boxes`` - each internal box is the min/max over its leaf range.

Node ids are canonical: internal k -> k, leaf k -> (n-1)+k, sentinel -> -1.
"""
from __future__ import annotations

import sys

import numpy as np

INF = sys.maxsize


def aug_keys(sorted_codes):
    """Keys augmented with their sorted position (Sec. 3.2), as Python ints."""
    return [(int(c) << 32) | i for i, c in enumerate(np.asarray(sorted_codes, dtype=np.uint64).tolist())]


def dstar_table(sorted_codes):
    """delta*(i) for i in [-1, n-1]: highest differing bit, +inf at both ends."""
    aug = aug_keys(sorted_codes)
    n = len(aug)
    d = {-1: INF, n - 1: INF}
    for i in range(n - 1):
        d[i] = (aug[i] ^ aug[i + 1]).bit_length() - 1
    return d


def radix_tree_bruteforce(sorted_codes):
    """{(l, r): split} for every internal node of the binary radix tree."""
    aug = aug_keys(sorted_codes)
    n = len(aug)
    out = {}
    if n < 2:
        return out
    work = [(0, n - 1)]
    while work:
        l, r = work.pop()
        if l == r:
            continue
        k = (aug[l] ^ aug[r]).bit_length() - 1
        g = l
        while g + 1 <= r and not (aug[g + 1] >> k) & 1:
            g += 1
        out[(l, r)] = g
        work.append((l, g))
        work.append((g + 1, r))
    return out


def check_karras_tree(sorted_codes, left, right, range_l=None, range_r=None, split=None):
    """Assert the Sec. 3.1 invariants; return (range_l, range_r, split) derived from left/right."""
    n = len(sorted_codes)
    ni = n - 1
    left = np.asarray(left).tolist()
    right = np.asarray(right).tolist()
    assert len(left) == max(ni, 0) and len(right) == max(ni, 0)
    if n < 2:
        return [], [], []
    # derive ranges top-down from the child links alone
    rl = [None] * ni
    rr = [None] * ni
    parent = [None] * ni
    rl[0], rr[0] = 0, n - 1
    seen_internal = {0}
    seen_leaf = set()
    work = [0]
    while work:
        k = work.pop()
        for side, c in (("L", left[k]), ("R", right[k])):
            assert -1 < c < 2 * n - 1, f"child id {c} out of range"
            if c >= ni:
                assert c - ni not in seen_leaf, "leaf reached twice"
                seen_leaf.add(c - ni)
            else:
                assert c not in seen_internal, "internal node reached twice"
                seen_internal.add(c)
                parent[c] = (k, side)
                work.append(c)
        lc, rc = left[k], right[k]
        # Karras numbering: a left child is numbered by its range end, a
        # right child by its range start (a leaf covers only itself)
        if lc < ni:
            rl[lc], rr[lc] = rl[k], lc
            lend = lc
        else:
            assert lc - ni == rl[k], "left leaf must be the range start"
            lend = lc - ni
        if rc < ni:
            rl[rc], rr[rc] = rc, rr[k]
            rbeg = rc
        else:
            assert rc - ni == rr[k], "right leaf must be the range end"
            rbeg = rc - ni
        assert rl[k] <= lend < rr[k], "split inside the range"
        assert rbeg == lend + 1, "children must be adjacent at the split"
    assert seen_internal == set(range(ni)), "every internal id exactly once"
    assert seen_leaf == set(range(n)), "every leaf exactly once"
    d = dstar_table(sorted_codes)
    splits = []
    for k in range(ni):
        l, r = rl[k], rr[k]
        assert k in (l, r), "node i's range starts or ends at i"
        lc = left[k]
        g = lc if lc < ni else lc - ni
        splits.append(g)
        # split = unique argmax of delta* over [l, r-1]
        inner = [d[j] for j in range(l, r)]
        assert d[g] == max(inner) and inner.count(d[g]) == 1
        # the index is the bound with the smaller delta* (root: left bound)
        expect = r if d[r] < d[l - 1] else l
        assert k == expect, f"node {k}: index rule gives {expect}"
    if range_l is not None:
        assert list(np.asarray(range_l)) == rl
        assert list(np.asarray(range_r)) == rr
    if split is not None:
        assert list(np.asarray(split)) == splits
    brute = radix_tree_bruteforce(sorted_codes)
    assert brute == {(rl[k], rr[k]): splits[k] for k in range(ni)}
    return rl, rr, splits


def preorder(n, left, right):
    ni = n - 1
    if n == 0:
        return []
    out, stack = [], [0]
    while stack:
        k = stack.pop()
        out.append(k)
        if k < ni:
            stack.append(int(right[k]))
            stack.append(int(left[k]))
    return out


def check_skips(sorted_codes, left, right, skip_internal, skip_leaf):
    n = len(sorted_codes)
    ni = n - 1
    if n == 0:
        return
    left = np.asarray(left).tolist()
    right = np.asarray(right).tolist()
    si = np.asarray(skip_internal).tolist()
    sl = np.asarray(skip_leaf).tolist()

    def skip(k):
        return sl[k - ni] if k >= ni else si[k]

    order = preorder(n, left, right)
    assert len(order) == 2 * n - 1
    # Algorithm 1 with an always-true predicate
    walk, leaves, node = [], [], 0
    while node != -1:
        walk.append(node)
        assert len(walk) <= 2 * n - 1, "walk does not terminate"
        if node >= ni:
            leaves.append(node - ni)
            node = skip(node)
        else:
            node = left[node]
    assert walk == order, "always-true walk must be the pre-order"
    assert leaves == list(range(n))
    # subtree sizes -> skip = pre-order successor past the subtree
    size = {}
    for k in reversed(order):
        size[k] = 1 if k >= ni else 1 + size[left[k]] + size[right[k]]
    pos = {k: i for i, k in enumerate(order)}
    for k in order:
        j = pos[k] + size[k]
        expect = order[j] if j < len(order) else -1
        assert skip(k) == expect, f"skip of {k}: {skip(k)} != {expect}"
    # Algorithm 2: closed form from the range end and delta*
    if n >= 2:
        rl, rr, _ = check_karras_tree(sorted_codes, left, right)
        d = dstar_table(sorted_codes)
        ends = {k: rr[k] for k in range(ni)}
        ends.update({ni + k: k for k in range(n)})
        for k, r in ends.items():
            if r == n - 1:
                expect = -1
            else:
                expect = ni + r + 1 if d[r] < d[r + 1] else r + 1
            assert skip(k) == expect


def check_boxes(n, range_l, range_r, leaf_box, internal_box):
    leaf_box = np.asarray(leaf_box, np.float32).reshape(n, 6)
    internal_box = np.asarray(internal_box, np.float32).reshape(-1, 6)
    for k in range(n - 1):
        seg = leaf_box[range_l[k]:range_r[k] + 1]
        expect = np.concatenate([seg[:, :3].min(axis=0), seg[:, 3:].max(axis=0)])
        assert np.array_equal(internal_box[k].view(np.uint32), expect.view(np.uint32)), f"box {k}"


def parse_node(name, n):
    """'I3' -> 3, 'L4' -> (n-1)+4, 'S' -> -1."""
    if name == "S":
        return -1
    k = int(name[1:])
    return k if name[0] == "I" else (n - 1) + k
