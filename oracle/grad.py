"""Oracle: the dual bound after T deferred-MMA iterations as a differentiable function of
the element costs, in plain PyTorch (FP64, CPU), differentiated by autograd.

Test infrastructure only (see ``oracle/__init__.py``). It computes exactly what
``oracle/solver.py`` computes (same readings: lambda^0 = c / |J|, pend = 0, omega,
b from one backward min-sum pass, forward then backward half-pass per iteration,
bound E(lambda + pend) + constant, Eq. D), written with tensor operations so that
autograd gives d bound / d c. The deferred schedule makes every BDD of a half-pass use
the previous half-pass's mean, so the layers at the same depth of all BDDs are processed
together; within a BDD the layers stay in order. Minima are ``scatter_reduce(amin)``;
autograd splits the gradient evenly between tied minima (a valid subgradient; at generic
costs there are no ties). Unreachable nodes carry a large finite cost BIG instead of
infinity so that no inf - inf enters the backward pass.

The bound is piecewise linear in c (min-plus operations and linear updates), so its
gradient is exact wherever it is differentiable.
"""
from __future__ import annotations

import numpy as np
import torch

from .bdd import BOT, TOP, Decomposition

BIG = 1e30


class _Depths:
    """Per direction and depth: the layers at that depth of every BDD long enough, their
    nodes, and where each node sits in the depth's node list."""

    def __init__(self, dec: Decomposition, forward: bool):
        blp = dec.bdd_layer_ptr
        lnp = dec.layer_node_ptr
        lengths = np.diff(blp)
        depth = int(lengths.max()) if len(lengths) else 0
        self.layers, self.nodes, self.seg = [], [], []
        self.pos = np.full(dec.n_nodes, -1, np.int64)  # node -> index within its depth's list
        for t in range(depth):
            js = np.nonzero(lengths > t)[0]
            ls = blp[js] + t if forward else blp[js + 1] - 1 - t
            counts = lnp[ls + 1] - lnp[ls]
            nodes = np.concatenate([np.arange(lnp[l], lnp[l + 1]) for l in ls])
            seg = np.repeat(np.arange(len(ls)), counts)
            self.pos[nodes] = np.arange(len(nodes))
            self.layers.append(torch.from_numpy(ls))
            self.nodes.append(torch.from_numpy(nodes))
            self.seg.append(torch.from_numpy(seg))


def _child_cost(b: torch.Tensor, c: torch.Tensor) -> torch.Tensor:
    """Cost from a child index: b[c] for a node, 0 for TOP, BIG for BOT."""
    val = b[c.clamp(min=0)]
    return torch.where(c >= 0, val, torch.where(c == TOP, torch.zeros_like(val), torch.full_like(val, BIG)))


def _seg_min(x: torch.Tensor, seg: torch.Tensor, n: int) -> torch.Tensor:
    return torch.full((n,), BIG, dtype=x.dtype).scatter_reduce(0, seg, x, "amin", include_self=True)


class UnrolledDual:
    """The deferred-MMA iteration on one decomposition, as tensor operations."""

    def __init__(self, dec: Decomposition, omega: float = 0.5):
        self.dec = dec
        self.omega = float(omega)
        self.fw = _Depths(dec, True)
        self.bw = _Depths(dec, False)
        self.lvar = torch.from_numpy(dec.layer_var)
        self.lo = torch.from_numpy(dec.node_lo)
        self.hi = torch.from_numpy(dec.node_hi)
        self.deg = torch.from_numpy(dec.deg).to(torch.float64)
        self.n_nodes = dec.n_nodes
        self.n_layers = dec.n_layers
        first = dec.bdd_layer_ptr[:-1]
        self.roots = torch.from_numpy(dec.layer_node_ptr[first])  # root node of every BDD

    # ---- passes ---------------------------------------------------------------------
    def _assemble(self, idx: list, vals: list, n: int) -> torch.Tensor:
        """Every index appears exactly once across the pieces."""
        i = torch.cat(idx)
        v = torch.cat(vals)
        return torch.zeros(n, dtype=v.dtype).index_put((i,), v)

    def backward_minsum(self, mu: torch.Tensor) -> torch.Tensor:
        """b of every node for per-layer costs mu (no update)."""
        b = torch.zeros(self.n_nodes, dtype=mu.dtype)
        idx, vals = [], []
        for t in range(len(self.bw.layers)):
            ls, nodes, seg = self.bw.layers[t], self.bw.nodes[t], self.bw.seg[t]
            v0 = _child_cost(b, self.lo[nodes])
            v1 = _child_cost(b, self.hi[nodes]) + mu[ls][seg]
            bt = torch.minimum(v0, v1)
            b = b.index_put((nodes,), bt)
            idx.append(nodes)
            vals.append(bt)
        return self._assemble(idx, vals, self.n_nodes)

    def forward_minima(self, mu: torch.Tensor) -> torch.Tensor:
        """Cheapest root -> TOP path cost of every BDD for per-layer costs mu."""
        f = torch.full((self.n_nodes,), BIG, dtype=mu.dtype).index_put((self.roots,), torch.zeros(len(self.roots),
                                                                                                  dtype=mu.dtype))
        top = torch.full((self.dec.nb,), BIG, dtype=mu.dtype)
        bdd_of_layer = torch.from_numpy(np.repeat(np.arange(self.dec.nb), np.diff(self.dec.bdd_layer_ptr)))
        for t in range(len(self.fw.layers)):
            ls, nodes, seg = self.fw.layers[t], self.fw.nodes[t], self.fw.seg[t]
            ft = f[nodes]
            w = mu[ls][seg]
            for child, add in ((self.lo[nodes], None), (self.hi[nodes], w)):
                val = ft if add is None else ft + add
                into = child >= 0
                f = f.scatter_reduce(0, child[into], val[into], "amin", include_self=True)
                at_top = child == TOP
                top = top.scatter_reduce(0, bdd_of_layer[ls][seg][at_top], val[at_top], "amin", include_self=True)
        return top

    def half_pass(self, lam: torch.Tensor, pend: torch.Tensor, other: torch.Tensor, forward: bool):
        """One deferred-MMA half-pass. Returns (lambda, pend, this direction's node costs)."""
        D = self.fw if forward else self.bw
        lam_idx, lam_vals, node_idx, node_vals = [], [], [], []
        acc = torch.zeros(len(self.deg), dtype=lam.dtype)
        if forward:
            cur = torch.full((self.n_nodes,), BIG, dtype=lam.dtype).index_put(
                (self.roots,), torch.zeros(len(self.roots), dtype=lam.dtype))
        else:
            cur = torch.zeros(self.n_nodes, dtype=lam.dtype)
        for t in range(len(D.layers)):
            ls, nodes, seg = D.layers[t], D.nodes[t], D.seg[t]
            n_l = len(ls)
            var = self.lvar[ls]
            mu = lam[ls] + pend[var]
            if forward:
                ft = cur[nodes]
                m0 = _seg_min(ft + _child_cost(other, self.lo[nodes]), seg, n_l)
                m1 = _seg_min(ft + _child_cost(other, self.hi[nodes]), seg, n_l) + mu
            else:
                ft = other[nodes]
                m0 = _seg_min(ft + _child_cost(cur, self.lo[nodes]), seg, n_l)
                m1 = _seg_min(ft + _child_cost(cur, self.hi[nodes]), seg, n_l) + mu
            removed = self.omega * (m1 - m0)
            lam_out = mu - removed
            acc = acc.index_add(0, var, removed)
            lam_idx.append(ls)
            lam_vals.append(lam_out)
            if forward:
                node_idx.append(nodes)
                node_vals.append(ft)
                w = lam_out[seg]
                for child, val in ((self.lo[nodes], ft), (self.hi[nodes], ft + w)):
                    into = child >= 0
                    cur = cur.scatter_reduce(0, child[into], val[into], "amin", include_self=True)
            else:
                v0 = _child_cost(cur, self.lo[nodes])
                v1 = _child_cost(cur, self.hi[nodes]) + lam_out[seg]
                bt = torch.minimum(v0, v1)
                cur = cur.index_put((nodes,), bt)
                node_idx.append(nodes)
                node_vals.append(bt)
        lam_new = self._assemble(lam_idx, lam_vals, self.n_layers)
        pend_new = torch.where(self.deg > 0, acc / self.deg.clamp(min=1), torch.zeros_like(acc))
        nodes_new = self._assemble(node_idx, node_vals, self.n_nodes)
        return lam_new, pend_new, nodes_new

    # ---- the differentiable bound --------------------------------------------------
    def lower_bound(self, cost: torch.Tensor, iters: int) -> torch.Tensor:
        """E(lambda + pend) + constant after `iters` iterations from lambda^0 = cost / |J|.

        `cost` has one entry per variable of the decomposition (original then auxiliary;
        auxiliary entries are 0 and fixed variables are not in any BDD). The constant is
        the cost of the variables presolve fixed to 1, passed in through `fixed_one`."""
        deg_l = self.deg[self.lvar]
        lam = cost[self.lvar] / deg_l
        pend = torch.zeros(len(self.deg), dtype=cost.dtype)
        b = self.backward_minsum(lam)
        for _ in range(iters):
            lam, pend, f = self.half_pass(lam, pend, b, True)
            lam, pend, b = self.half_pass(lam, pend, f, False)
        return self.forward_minima(lam + pend[self.lvar]).sum()


def bound_and_grad(dec: Decomposition, cost: np.ndarray, fixed: np.ndarray, iters: int, omega: float = 0.5):
    """(bound, d bound / d cost) for element costs `cost` (one per variable of (P)).

    Variables fixed to 1 by presolve add their cost to the bound (gradient 1), variables
    fixed to 0 have gradient 0, free variables get the adjoint of the unrolled iteration."""
    c = torch.tensor(np.concatenate([cost, np.zeros(dec.nvars_total - dec.nvars)]), dtype=torch.float64,
                     requires_grad=True)
    ud = UnrolledDual(dec, omega)
    one = torch.from_numpy(np.concatenate([fixed == 1, np.zeros(dec.nvars_total - dec.nvars, bool)]))
    lb = ud.lower_bound(c, iters) + (c * one).sum()
    lb.backward()
    return float(lb.detach()), c.grad.numpy()[: dec.nvars].copy()
