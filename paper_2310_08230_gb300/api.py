"""NumPy / PyTorch wrapper of the C ABI (argument marshalling only; every step runs in the
CUDA library).

    d = pair_costs(FX, FY)                       # torch CUDA tensors -> (nvx, nvy) costs
    allowed = candidates(d, k, TX, TY)           # top-k pruned candidate mask (device)
    s = Solver(TX, TY, d, allowed)               # host compiler + device BDD store
    s.dual(200); lb = s.lower_bound()            # deferred min-marginal averaging, Eq. D
    x, cost = s.primal()                         # feasible matching by rounding
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L


def _torch():
    import torch

    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _mesh(T: np.ndarray, nv: int, V: np.ndarray | None = None):
    """disco_mesh over host arrays; returns (mesh, arrays to keep alive)."""
    T = np.ascontiguousarray(T, dtype=np.int32)
    Vp = None
    if V is not None:
        V = np.ascontiguousarray(V, dtype=np.float32)
        Vp = V.ctypes.data_as(ctypes.c_void_p)
    m = L.disco_mesh(int(nv), int(T.shape[0]), Vp, T.ctypes.data_as(ctypes.c_void_p))
    return m, (T, V)


def _ptr(a) -> int:
    """Data pointer of a NumPy array or a torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())


def pair_costs(FX, FY, stream=None):
    """d[m, n] = mean_k (FX[m, k] - FY[n, k])^2 (FP32, CUDA tensors in and out)."""
    torch = _torch()
    FX = FX.contiguous().float()
    FY = FY.contiguous().float()
    d = torch.empty((FX.shape[0], FY.shape[0]), dtype=torch.float32, device=FX.device)
    L.check(L.lib().disco_pair_costs(FX.data_ptr(), FY.data_ptr(), FX.shape[0], FY.shape[0], FX.shape[1],
                                     d.data_ptr(), _stream_ptr(stream)), "disco_pair_costs")
    return d


def pair_distances(FX, FY, stream=None):
    """d[m, n] = ||FX[m] - FY[n]|| (FP32, CUDA tensors in and out), the feature distance of Eq. 2."""
    torch = _torch()
    FX = FX.contiguous().float()
    FY = FY.contiguous().float()
    d = torch.empty((FX.shape[0], FY.shape[0]), dtype=torch.float32, device=FX.device)
    L.check(L.lib().disco_pair_distances(FX.data_ptr(), FY.data_ptr(), FX.shape[0], FY.shape[0], FX.shape[1],
                                         d.data_ptr(), _stream_ptr(stream)), "disco_pair_distances")
    return d


def candidates(d, k: int, TX: np.ndarray, TY: np.ndarray, stream=None):
    """Top-k candidate mask widened by closed 1-rings (uint8 CUDA tensor, nvx x nvy)."""
    torch = _torch()
    nvx, nvy = int(d.shape[0]), int(d.shape[1])
    mx, tx = _mesh(TX, nvx)
    my, ty = _mesh(TY, nvy)
    allowed = torch.empty((nvx, nvy), dtype=torch.uint8, device=d.device)
    L.check(L.lib().disco_candidates(d.contiguous().data_ptr(), nvx, nvy, int(k), ctypes.byref(mx), ctypes.byref(my),
                                     allowed.data_ptr(), _stream_ptr(stream)), "disco_candidates")
    return allowed


def candidates_coarse_to_fine(pairs: np.ndarray, c2f_x: np.ndarray, c2f_y: np.ndarray, rings: int,
                              TX: np.ndarray, nvx: int, TY: np.ndarray, nvy: int) -> np.ndarray:
    """Fine candidate mask (uint8, nvx x nvy) around the coarse vertex pairs `pairs` (k x 2):
    pairs within `rings` edges, on both fine meshes, of a coarse match mapped by c2f_x / c2f_y."""
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    cx = np.ascontiguousarray(c2f_x, dtype=np.int32)
    cy = np.ascontiguousarray(c2f_y, dtype=np.int32)
    mx, kx = _mesh(TX, nvx)
    my, ky = _mesh(TY, nvy)
    out = np.zeros((nvx, nvy), np.uint8)
    L.check(L.lib().disco_candidates_coarse_to_fine(pairs.ctypes.data, pairs.shape[0], cx.ctypes.data, cx.shape[0],
                                                    cy.ctypes.data, cy.shape[0], int(rings), ctypes.byref(mx),
                                                    ctypes.byref(my), out.ctypes.data), "disco_candidates_coarse_to_fine")
    return out


def solve_coarse_to_fine(levels, costs, rings: int = 1, iters: int = 100, **opts) -> list[dict]:
    """Coarse-to-fine solving (Sec. 4): the coarsest level on its full product space, every
    finer level on the candidates within `rings` edges of the previous level's matching.

    levels: [(TX, TY, c2f_x, c2f_y)] from coarse to fine, c2f_* mapping a level's vertex ids
    to the next level's (ignored at the finest); costs: per level the (nvx, nvy) pair costs.
    Returns per level: bound, matching x, its cost, feasibility, the vertex pairs of the
    matching and the candidate density used."""
    out = []
    allowed = None
    for k, ((TX, TY, cx, cy), d) in enumerate(zip(levels, costs)):
        nvx, nvy = int(d.shape[0]), int(d.shape[1])
        s = Solver(TX, TY, d, allowed, **opts)
        s.dual(iters)
        lb = s.lower_bound()
        x, cost, ok = s.primal()
        pairs = s.point_map(x)
        s.close()
        out.append({"lower_bound": lb, "x": x, "cost": cost, "feasible": ok, "pairs": pairs,
                    "density": 1.0 if allowed is None else float(np.mean(allowed))})
        if not ok:
            break
        if k + 1 < len(levels):
            nTX, nTY = levels[k + 1][0], levels[k + 1][1]
            nd = costs[k + 1]
            allowed = candidates_coarse_to_fine(pairs, cx, cy, rings, nTX, int(nd.shape[0]), nTY, int(nd.shape[1]))
    return out


def balanced_groups(weights, groups: int) -> list[list[int]]:
    """Indices 0 .. n-1 split into at most ``groups`` groups of about equal total weight:
    heaviest first onto the lightest group (ties to the lower group), each group in
    ascending index order, empty groups dropped."""
    n = len(weights)
    g = max(1, min(int(groups), n))
    load = [0.0] * g
    members = [[] for _ in range(g)]
    for i in sorted(range(n), key=lambda i: -weights[i]):
        k = min(range(g), key=lambda k: load[k])
        members[k].append(i)
        load[k] += weights[i]
    return [sorted(m) for m in members if m]


def solve_batch_pipelined(pairs, iters: int, groups: int = 2, weights=None, **opts) -> list[dict]:
    """Many pairs as ``groups`` batched handles, pipelined between host and GPU.

    ``pairs`` as for :meth:`Solver.batch`. The pairs are split into groups of about equal
    ``weights`` (default: the size of each pair's cost matrix), largest first onto the
    lightest group. Each group is one batched device store on its own stream: the host
    compiles group g + 1 while the GPU runs the ``iters`` dual iterations of group g (their
    graph replays are only enqueued), then every group is rounded. The lower bounds are
    those of one batch over all pairs, bit for bit (each pair's bound is summed in its own
    fixed order). A batch build compiles its pairs side by side on the host threads, so
    small groups compile less efficiently; two groups suit batches of a few dozen pairs on
    16 cores. Returns per pair, in input order: lower_bound, x, cost, feasible. The
    launch-geometry autotuner is off unless ``autotune`` is given: its timed trials would
    wait behind the previous group's iterations (every geometry gives the same results)."""
    torch = _torch()
    opts.setdefault("autotune", 0)
    n = len(pairs)
    w = [float(np.prod(p[2].shape)) for p in pairs] if weights is None else [float(x) for x in weights]
    members = balanced_groups(w, groups)
    streams = [torch.cuda.Stream() for _ in members]
    torch.cuda.synchronize()  # inputs computed on other streams are complete
    solvers = []
    try:
        for m, st in zip(members, streams):
            s = Solver.batch([pairs[i] for i in m], stream=int(st.cuda_stream), **opts)
            solvers.append(s)
            s.dual(iters)  # enqueued: runs while the next group compiles
        out = [None] * n
        for m, s in zip(members, solvers):
            lbs = s.lower_bounds()
            xs, costs, ok = s.primal_batch()
            for j, i in enumerate(m):
                out[i] = {"lower_bound": float(lbs[j]), "x": xs[j], "cost": float(costs[j]), "feasible": bool(ok[j])}
        return out
    finally:
        for s in solvers:
            s.close()


def default_opts(**kw) -> L.disco_opts:
    o = L.disco_opts()
    L.check(L.lib().disco_default_opts(ctypes.byref(o)), "disco_default_opts")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class Solver:
    """One shape pair: ILP (P) compiled to BDDs and solved by the GPU dual / primal."""

    def __init__(self, TX: np.ndarray, TY: np.ndarray, d, allowed=None, nvx: int | None = None,
                 nvy: int | None = None, VX=None, VY=None, **opts):
        nvx = int(d.shape[0]) if nvx is None else nvx
        nvy = int(d.shape[1]) if nvy is None else nvy
        if isinstance(d, np.ndarray):
            d = np.ascontiguousarray(d, dtype=np.float32)
        if isinstance(allowed, np.ndarray):
            allowed = np.ascontiguousarray(allowed, dtype=np.uint8)
        mx, self._tx = _mesh(TX, nvx, VX)
        my, self._ty = _mesh(TY, nvy, VY)
        self.opts = default_opts(**opts)
        h = ctypes.c_void_p()
        L.check(L.lib().disco_build(ctypes.byref(mx), ctypes.byref(my), _ptr(d),
                                    None if allowed is None else _ptr(allowed), ctypes.byref(self.opts),
                                    ctypes.byref(h)), "disco_build")
        self.h = h
        self._sizes = [(nvx, nvy)]

    # -------------------------------------------------------------------------------
    def info(self) -> dict:
        i = L.disco_info_t()
        L.check(L.lib().disco_info(self.h, ctypes.byref(i)), "disco_info")
        return {k: getattr(i, k) for k, _ in i._fields_ if k != "reserved"}

    def dual(self, iters: int) -> None:
        L.check(L.lib().disco_dual(self.h, int(iters)), "disco_dual")

    def dual_qn(self, calls: int, mma_iters: int = 20) -> None:
        """`calls` quasi-Newton powered iterations (Alg. 1), each with `mma_iters` MMA iterations."""
        L.check(L.lib().disco_dual_qn(self.h, int(calls), int(mma_iters)), "disco_dual_qn")

    def lower_bound(self) -> float:
        lb = ctypes.c_double()
        L.check(L.lib().disco_lower_bound(self.h, ctypes.byref(lb)), "disco_lower_bound")
        return lb.value

    def converge(self, max_iters: int) -> tuple[int, float, bool]:
        n = ctypes.c_int32()
        lb = ctypes.c_double()
        rc = L.lib().disco_converge(self.h, int(max_iters), ctypes.byref(n), ctypes.byref(lb))
        if rc not in (L.DISCO_OK, L.DISCO_ERR_TIMEOUT):
            L.check(rc, "disco_converge")
        return n.value, lb.value, rc == L.DISCO_OK

    def min_marginals(self, out=None) -> np.ndarray:
        ns = self.info()["nslots"]
        if out is None:
            out = np.empty(ns, np.float32)
        L.check(L.lib().disco_min_marginals(self.h, _ptr(out), int(out.shape[0])), "disco_min_marginals")
        return out

    def primal(self) -> tuple[np.ndarray, float, bool]:
        nv = self.info()["nvars"]
        x = np.zeros(nv, np.uint8)
        c = ctypes.c_double()
        rc = L.lib().disco_primal(self.h, x.ctypes.data, nv, ctypes.byref(c))
        if rc not in (L.DISCO_OK, L.DISCO_ERR_PRIMAL_FAILED):
            L.check(rc, "disco_primal")
        return x, c.value, rc == L.DISCO_OK

    def point_map(self, x: np.ndarray) -> np.ndarray:
        """Vertex pairs (k x 2, sorted) at the corners of the matching elements set in x."""
        x = np.ascontiguousarray(x, dtype=np.uint8)
        n = ctypes.c_int64()
        cap = 3 * int(x.sum()) + 1
        out = np.zeros((cap, 2), np.int32)
        L.check(L.lib().disco_point_map(self.h, x.ctypes.data, x.shape[0], out.ctypes.data, cap, ctypes.byref(n)),
                "disco_point_map")
        return out[: n.value].copy()

    def get_state(self) -> tuple[np.ndarray, np.ndarray]:
        inf = self.info()
        lam = np.empty(inf["nslots"], np.float32)
        pend = np.empty(inf["nvars_free"] + inf["nvars_aux"], np.float32)
        L.check(L.lib().disco_get_state(self.h, lam.ctypes.data, lam.shape[0], pend.ctypes.data, pend.shape[0]),
                "disco_get_state")
        return lam, pend

    def set_state(self, lam: np.ndarray, pend: np.ndarray | None = None) -> None:
        lam = np.ascontiguousarray(lam, np.float32)
        pp = None if pend is None else np.ascontiguousarray(pend, np.float32)
        L.check(L.lib().disco_set_state(self.h, lam.ctypes.data, lam.shape[0],
                                        None if pp is None else pp.ctypes.data, 0 if pp is None else pp.shape[0]),
                "disco_set_state")

    def record(self, iters: int, checkpoint_every: int = 10) -> None:
        """Restart at lambda^0 and run `iters` iterations keeping checkpoints for grad()."""
        L.check(L.lib().disco_record(self.h, int(iters), int(checkpoint_every)), "disco_record")

    def grad(self, out=None):
        """d(bound after the recorded iterations) / d(pair costs): (nvx, nvy) per instance,
        concatenated (float32; NumPy array, or `out`, a host or device buffer)."""
        n = self.pair_cost_count()
        if out is None:
            out = np.empty(n, np.float32)
        L.check(L.lib().disco_grad(self.h, _ptr(out), int(out.numel() if hasattr(out, "numel") else out.size)),
                "disco_grad")
        return out

    def pair_cost_count(self) -> int:
        return sum(a * b for a, b in self._sizes)

    @classmethod
    def batch(cls, pairs, **opts) -> "Solver":
        """One handle over several pairs: ``pairs`` = [(TX, TY, d, allowed_or_None[, VX, VY]), ...]."""
        self = cls.__new__(cls)
        n = len(pairs)
        meshes_x = (L.disco_mesh * n)()
        meshes_y = (L.disco_mesh * n)()
        keep = []
        dptr = (ctypes.c_void_p * n)()
        aptr = (ctypes.c_void_p * n)()
        for i, pair in enumerate(pairs):
            TX, TY, d, allowed = pair[:4]
            VX, VY = (pair[4], pair[5]) if len(pair) > 4 else (None, None)
            if isinstance(d, np.ndarray):
                d = np.ascontiguousarray(d, dtype=np.float32)
            if isinstance(allowed, np.ndarray):
                allowed = np.ascontiguousarray(allowed, dtype=np.uint8)
            mx, tx = _mesh(TX, int(d.shape[0]), VX)
            my, ty = _mesh(TY, int(d.shape[1]), VY)
            meshes_x[i] = mx
            meshes_y[i] = my
            dptr[i] = _ptr(d)
            aptr[i] = None if allowed is None else _ptr(allowed)
            keep += [tx, ty, d, allowed]
        self.opts = default_opts(**opts)
        h = ctypes.c_void_p()
        L.check(L.lib().disco_build_batch(n, meshes_x, meshes_y, ctypes.cast(dptr, ctypes.c_void_p),
                                          ctypes.cast(aptr, ctypes.c_void_p), ctypes.byref(self.opts),
                                          ctypes.byref(h)), "disco_build_batch")
        self.h = h
        self._keep = keep
        self._sizes = [(int(p[2].shape[0]), int(p[2].shape[1])) for p in pairs]
        return self

    def batch_size(self) -> int:
        n = ctypes.c_int32()
        L.check(L.lib().disco_batch_size(self.h, ctypes.byref(n)), "disco_batch_size")
        return n.value

    def lower_bounds(self) -> np.ndarray:
        n = self.batch_size()
        out = np.zeros(n, np.float64)
        L.check(L.lib().disco_lower_bounds(self.h, out.ctypes.data_as(L.c_double_p), n), "disco_lower_bounds")
        return out

    def instance_info(self, i: int) -> dict:
        inf = L.disco_info_t()
        L.check(L.lib().disco_instance_info(self.h, int(i), ctypes.byref(inf)), "disco_instance_info")
        return {k: getattr(inf, k) for k, _ in inf._fields_ if k != "reserved"}

    def primal_batch(self) -> tuple[list, np.ndarray, np.ndarray]:
        """Per pair: (x_i, cost_i, feasible_i)."""
        n = self.batch_size()
        sizes = [self.instance_info(i)["nvars"] for i in range(n)]
        x = np.zeros(sum(sizes), np.uint8)
        costs = np.zeros(n, np.float64)
        status = np.zeros(n, np.int32)
        rc = L.lib().disco_primal_batch(self.h, x.ctypes.data, x.shape[0], costs.ctypes.data_as(L.c_double_p),
                                        status.ctypes.data_as(L.c_int32_p), n)
        if rc not in (L.DISCO_OK, L.DISCO_ERR_PRIMAL_FAILED):
            L.check(rc, "disco_primal_batch")
        xs = np.split(x, np.cumsum(sizes)[:-1])
        return xs, costs, status == 0

    def close(self) -> None:
        if getattr(self, "h", None):
            L.lib().disco_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
