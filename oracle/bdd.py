"""Oracle: constraint -> BDD compilation and BDD splitting.

Plain Python, explicit node graphs. Test infrastructure only (see
``oracle/__init__.py``).

* BDD definition (App. A.3, "Constraint Splitting"): layered DAG, one layer per
  variable, a 0-arc and a 1-arc per node, arcs only from one layer to the next
  or to a terminal (no skipping arcs), a unique root, reduced.
* A linear row sum_l a_l x_l = r is compiled by its partial sums: the nodes of
  layer l are the partial sums of the first l variables that are reachable from
  the root AND from which r is still reachable (Sec. 3.2 "Constraint
  Splitting"; Fig. BDD shows sum_{i<=8} x_i = 2 with 20 nodes).
* Splitting (App. A.3, Alg. 3, Fig. BDD): cut after some layer; if the next
  layer has k nodes, add auxiliary variables y_1..y_k with y_j = 1 iff the j-th
  node of that layer (ascending partial sum) is used. The left part ends with a
  chain over y_1..y_k that forces exactly that y_j; the right part starts with
  a chain over y_1..y_k that reads it and enters node j.

Readings: a cut whose next layer has a single node needs no auxiliary variable
(both parts share no variable); segments are balanced: a row of n layers with
chunk c > 0 and n > c is cut into S = min(ceil(n/c), K) segments at layers
floor(s n / S), K = the segment cap (0 = none). The cap keeps very long rows in
few segments: a one-hot chain carries cost information across one cut per
half-pass.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BOT = -1
TOP = -2


@dataclass
class BDD:
    """Layer l tests variable ``var[l]``; ``lo[l][u]`` / ``hi[l]][u]`` is the index of the child
    in layer l+1, or BOT / TOP. Layer 0 has exactly one node (the root)."""

    var: list = field(default_factory=list)
    lo: list = field(default_factory=list)
    hi: list = field(default_factory=list)

    @property
    def n_layers(self) -> int:
        return len(self.var)

    def widths(self) -> list:
        return [len(x) for x in self.lo]

    def n_nodes(self) -> int:
        return sum(self.widths())

    def evaluate(self, assign: dict) -> bool:
        """True iff the path selected by ``assign`` (var -> 0/1) ends in TOP."""
        u = 0
        for l in range(self.n_layers):
            c = self.hi[l][u] if assign[self.var[l]] else self.lo[l][u]
            if c == BOT:
                return False
            if c == TOP:
                return l == self.n_layers - 1
            u = c
        return False


def compile_row(vars_: np.ndarray, coefs: np.ndarray, rhs: int) -> tuple[BDD, list]:
    """Reduced BDD of sum_l coefs[l] x_{vars[l]} = rhs (variables in the given order).

    Also returns the partial sum of every node, per layer (ascending)."""
    n = len(vars_)
    a_all = [int(c) for c in coefs]
    # largest amount the layers l.. can still add (p_rem) or subtract (q_rem)
    p_rem = [0] * (n + 1)
    q_rem = [0] * (n + 1)
    for l in range(n - 1, -1, -1):
        p_rem[l] = p_rem[l + 1] + (a_all[l] > 0)
        q_rem[l] = q_rem[l + 1] + (a_all[l] < 0)
    # forward: partial sums reachable from the root (sums that could never come back
    # to rhs are dropped early; the backward pass below would drop them anyway)
    reach = [{0}]
    for l in range(n):
        a = a_all[l]
        nxt = {s for s in reach[l]} | {s + a for s in reach[l]}
        reach.append({s for s in nxt if -q_rem[l + 1] <= rhs - s <= p_rem[l + 1]})
    keep = [None] * (n + 1)
    keep[n] = {rhs} & reach[n]
    for l in range(n - 1, -1, -1):
        a = int(coefs[l])
        keep[l] = {s for s in reach[l] if (s in keep[l + 1]) or (s + a in keep[l + 1])}
    if not keep[0]:
        raise ValueError("infeasible row")
    sums = [sorted(k) for k in keep[:n]]
    bdd = BDD()
    for l in range(n):
        a = int(coefs[l])
        nxt = {s: j for j, s in enumerate(sorted(keep[l + 1]))} if l + 1 < n else None
        lo, hi = [], []
        for s in sums[l]:
            for target, out in ((s, lo), (s + a, hi)):
                if l + 1 < n:
                    out.append(nxt.get(target, BOT))
                else:
                    out.append(TOP if target == rhs else BOT)
        bdd.var.append(int(vars_[l]))
        bdd.lo.append(lo)
        bdd.hi.append(hi)
    return bdd, sums


def split(bdd: BDD, cut: int, aux_ids: list | None) -> tuple[BDD, BDD]:
    """Alg. 3: split after layer ``cut - 1`` (the right part starts at layer ``cut``).

    ``aux_ids`` are the k variable ids y_1..y_k (k = width of layer ``cut``), or None
    when that layer has a single node."""
    k = len(bdd.lo[cut])
    left = BDD(bdd.var[:cut], [list(x) for x in bdd.lo[:cut]], [list(x) for x in bdd.hi[:cut]])
    right = BDD(bdd.var[cut:], [list(x) for x in bdd.lo[cut:]], [list(x) for x in bdd.hi[cut:]])
    if k == 1:
        assert aux_ids is None
        # arcs into the single node of layer ``cut`` now end in TOP
        for arr in (left.lo[cut - 1], left.hi[cut - 1]):
            for u, c in enumerate(arr):
                if c == 0:
                    arr[u] = TOP
        return left, right
    assert aux_ids is not None and len(aux_ids) == k
    # ---- left part: arcs into node w of layer ``cut`` go to state "exit w" of the y_1 layer.
    # States of the y_j layer: j == 1: [exit 0 .. exit k-1];
    #                          j >= 2: [chosen, exit j-1 .. exit k-1]  (0-based exits).
    def left_state(j: int, exit_: int | None) -> int:
        if j == 1:
            return exit_
        return 0 if exit_ is None else 1 + exit_ - (j - 1)

    for j in range(1, k + 1):
        width = k if j == 1 else k - j + 2
        lo, hi = [BOT] * width, [BOT] * width
        states = [(None if (j >= 2 and u == 0) else (u if j == 1 else u - 1 + (j - 1))) for u in range(width)]
        for u, ex in enumerate(states):
            if ex is None:  # already chosen: every later y must be 0
                lo[u] = TOP if j == k else left_state(j + 1, None)
            elif ex == j - 1:  # the exit node is the j-th: y_j must be 1
                hi[u] = TOP if j == k else left_state(j + 1, None)
            else:  # exit further on: y_j must be 0
                lo[u] = left_state(j + 1, ex)
        left.var.append(aux_ids[j - 1])
        left.lo.append(lo)
        left.hi.append(hi)
    # ---- right part: states of the y_j layer: [pending, chosen 0 .. chosen j-2]
    pre = BDD()
    for j in range(1, k + 1):
        width = j
        lo, hi = [BOT] * width, [BOT] * width
        for u in range(width):
            if u == 0:  # nothing chosen yet
                if j < k:
                    lo[u] = 0
                    hi[u] = j  # chosen j-1 (0-based) sits at index j in the next layer
                else:
                    hi[u] = k - 1  # y_k must be 1: enter node k-1
            else:  # chosen u-1 already: y_j must be 0
                lo[u] = u if j < k else u - 1
        pre.var.append(aux_ids[j - 1])
        pre.lo.append(lo)
        pre.hi.append(hi)
    right = BDD(pre.var + right.var, pre.lo + right.lo, pre.hi + right.hi)
    return left, right


def segment_bounds(n: int, chunk: int, max_segments: int = 8) -> list:
    """Layer indices where segments start (balanced), plus n."""
    if chunk <= 0 or n <= chunk:
        return [0, n]
    nseg = -(-n // chunk)
    if max_segments > 0:
        nseg = min(nseg, max_segments)
    return [(s * n) // nseg for s in range(nseg + 1)]


def split_row(bdd: BDD, chunk: int, next_aux: int, max_segments: int = 8) -> tuple[list, list, int]:
    """Cut a row's BDD into balanced segments. Returns (segments, aux var ids, next free id).

    Auxiliary ids are handed out cut by cut (left to right), y_1..y_k within a cut."""
    bounds = segment_bounds(bdd.n_layers, chunk, max_segments)
    segs = []
    aux = []
    rest = bdd
    consumed = 0  # original layers already cut off the front of ``rest``
    prefix = 0  # auxiliary prefix layers at the front of ``rest``
    for s in range(1, len(bounds) - 1):
        cut_orig = bounds[s]
        cut = prefix + (cut_orig - consumed)
        k = len(rest.lo[cut])
        ids = None
        if k > 1:
            ids = list(range(next_aux, next_aux + k))
            next_aux += k
            aux += ids
        left, rest = split(rest, cut, ids)
        segs.append(left)
        consumed = cut_orig
        prefix = k if k > 1 else 0
    segs.append(rest)
    return segs, aux, next_aux


@dataclass
class Decomposition:
    """All BDDs of the free part of (P), flattened for the numeric core."""

    nvars: int  # original variables
    nvars_total: int  # original + auxiliary
    bdd_row: np.ndarray  # row of (P) each BDD comes from
    bdd_layer_ptr: np.ndarray  # (nb+1,)
    layer_var: np.ndarray  # (nL,)
    layer_node_ptr: np.ndarray  # (nL+1,)
    node_lo: np.ndarray  # global child node index, BOT or TOP
    node_hi: np.ndarray
    deg: np.ndarray  # |J_i| over all BDDs (0 for fixed variables)
    cost: np.ndarray  # (nvars_total,) FP64, auxiliary variables cost 0
    free: np.ndarray  # bool (nvars,) not fixed by presolve
    const: float
    bdds: list

    @property
    def nb(self) -> int:
        return len(self.bdd_row)

    @property
    def n_layers(self) -> int:
        return len(self.layer_var)

    @property
    def n_nodes(self) -> int:
        return int(self.layer_node_ptr[-1])


def flatten(bdds: list, rows: list, nvars: int, nvars_total: int, cost: np.ndarray, free: np.ndarray,
            const: float) -> Decomposition:
    blp = [0]
    lvar, lnp, nlo, nhi = [], [0], [], []
    for b in bdds:
        for l in range(b.n_layers):
            base_next = lnp[-1] + len(b.lo[l])
            lvar.append(b.var[l])
            for c0, c1 in zip(b.lo[l], b.hi[l]):
                nlo.append(c0 if c0 < 0 else base_next + c0)
                nhi.append(c1 if c1 < 0 else base_next + c1)
            lnp.append(base_next)
        blp.append(len(lvar))
    lvar = np.array(lvar, np.int64)
    deg = np.bincount(lvar, minlength=nvars_total).astype(np.int64)
    return Decomposition(nvars, nvars_total, np.array(rows, np.int64), np.array(blp, np.int64), lvar,
                         np.array(lnp, np.int64), np.array(nlo, np.int64), np.array(nhi, np.int64), deg,
                         cost, free, const, bdds)


def decompose(prob, fixed: np.ndarray, const: float, chunk: int = 0, max_segments: int = 8) -> Decomposition:
    """Compile every row that still has free variables (after presolve) into BDD segments.

    Fixed variables are substituted into the right-hand side. Rows keep their order
    in (P); a row's segments are consecutive; auxiliary variables are numbered after
    the original ones."""
    bdds, rows = [], []
    next_aux = prob.nvars
    for r in range(prob.nrows):
        v, a, rhs = prob.row(r)
        f = fixed[v]
        rr = rhs - int(np.sum(a[f >= 0] * f[f >= 0]))
        sel = f < 0
        if not sel.any():
            assert rr == 0
            continue
        bdd, _ = compile_row(v[sel], a[sel], rr)
        segs, _aux, next_aux = split_row(bdd, chunk, next_aux, max_segments)
        bdds += segs
        rows += [r] * len(segs)
    cost = np.concatenate([prob.cost, np.zeros(next_aux - prob.nvars)])
    return flatten(bdds, rows, prob.nvars, next_aux, cost, fixed < 0, const)
