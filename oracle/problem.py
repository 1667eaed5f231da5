"""Oracle: costs, candidate pruning, product space and the constraint matrix of ILP (P).

Plain NumPy, FP64. Test infrastructure only (see ``oracle/__init__.py``).

Paper passages followed:
* product space of triangle-triangle, triangle-edge and triangle-vertex
  matching elements, at least one triangle in every element (Sec. 3.1, Fig. 2);
* closedness ("geometric consistency") rows  A^d x = 0 and projection rows
  A^M x = 1, A^N x = 1 of ILP (P) (Sec. 3.1, Eq. P);
* problem size about 21 |T_M||T_N| (App. B, Fig. runtime caption);
* cost: the configs replace Eq. 2 by the mean squared feature distance over
  the three vertex pairs, normalised to [0, 1] (Sec. 3.3, Eq. 2 variant);
* pruning to neighbourhoods of vertex matches (Sec. 4 coarse-to-fine, App.).

Readings where the paper is silent (each with its reason):
* element enumeration and canonical variable order: type (tri-tri,
  X-tri x Y-edge, X-edge x Y-tri, X-tri x Y-vertex, X-vertex x Y-tri), then the
  X element index, the Y element index, then rotation / pattern;
* a closedness row per product edge (unordered pair of product vertices whose
  X parts form an edge or one vertex and Y parts likewise, not both single
  vertices); an element adds +1 when it traverses the edge from its
  lexicographically smaller product vertex to the larger one, -1 otherwise;
* candidates: the k feature-nearest vertices of each vertex on the other mesh,
  widened by their closed 1-ring on that mesh (in both directions); an element is
  kept iff its three vertex pairs are allowed.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# vertex sequences of a degenerate (edge) triangle over an edge {a < b}: 0 -> a, 1 -> b
EDGE_PATTERNS = np.array([[0, 0, 1], [0, 1, 0], [1, 0, 0], [0, 1, 1], [1, 0, 1], [1, 1, 0]], dtype=np.int64)

TT, XT_YE, XE_YT, XT_YV, XV_YT = 0, 1, 2, 3, 4


def mesh_edges(T: np.ndarray) -> np.ndarray:
    """Undirected edges (a < b), sorted lexicographically."""
    T = np.asarray(T, dtype=np.int64)
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0)


def check_mesh(nv: int, T: np.ndarray) -> int:
    """Closed, consistently oriented 2-manifold check. Returns the Euler characteristic."""
    T = np.asarray(T, dtype=np.int64)
    if T.size == 0 or T.min() < 0 or T.max() >= nv:
        raise ValueError("triangle index out of range")
    directed = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    if np.any(directed[:, 0] == directed[:, 1]):
        raise ValueError("degenerate triangle")
    # every directed edge once, and its reverse exactly once
    u, cnt = np.unique(directed, axis=0, return_counts=True)
    if np.any(cnt != 1):
        raise ValueError("non-manifold or inconsistently oriented mesh")
    rev = {tuple(x) for x in u}
    for a, b in u:
        if (b, a) not in rev:
            raise ValueError("open mesh (boundary edge)")
    E = len(u) // 2
    used = np.unique(T).size
    if used != nv:
        raise ValueError("isolated vertex")
    return nv - E + len(T)


def pair_distance(FX: np.ndarray, FY: np.ndarray) -> np.ndarray:
    """d(m, n) = mean over feature dimensions of (F_X[m] - F_Y[n])^2, FP64 (Eq. 2 variant)."""
    FX = np.asarray(FX, dtype=np.float64)
    FY = np.asarray(FY, dtype=np.float64)
    diff = FX[:, None, :] - FY[None, :, :]
    return np.mean(diff * diff, axis=2)


def pair_euclid(FX: np.ndarray, FY: np.ndarray) -> np.ndarray:
    """d(m, n) = ||F_X[m] - F_Y[n]||, FP64 (the feature distance of Eq. 2)."""
    FX = np.asarray(FX, dtype=np.float64)
    FY = np.asarray(FY, dtype=np.float64)
    diff = FX[:, None, :] - FY[None, :, :]
    return np.sqrt(np.sum(diff * diff, axis=2))


def mixed_areas(V: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Mixed area of every vertex (Eq. 2's A; Meyer et al. 2003, "mixed area" of a vertex's
    1-ring). Per triangle: if no angle exceeds 90 degrees, corner P takes its Voronoi part
    (|PR|^2 cot Q + |PQ|^2 cot R) / 8; otherwise the obtuse corner takes half the triangle's
    area and the two others a quarter each."""
    V = np.asarray(V, dtype=np.float64)
    T = np.asarray(T, dtype=np.int64)
    out = np.zeros(len(V))
    for t in T:
        P = V[t]
        area = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
        if area == 0.0:
            continue
        # angle at each corner from the law of cosines on the opposite side
        ang = np.empty(3)
        for v in range(3):
            a, b = P[(v + 1) % 3] - P[v], P[(v + 2) % 3] - P[v]
            ang[v] = np.arccos(np.clip(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)), -1.0, 1.0))
        if ang.max() <= np.pi / 2:
            for v in range(3):
                q, r = (v + 1) % 3, (v + 2) % 3
                pr2 = np.sum((P[v] - P[r]) ** 2)
                pq2 = np.sum((P[v] - P[q]) ** 2)
                out[t[v]] += (pr2 / np.tan(ang[q]) + pq2 / np.tan(ang[r])) / 8.0
        else:
            ob = int(np.argmax(ang))
            for v in range(3):
                out[t[v]] += area / 2.0 if v == ob else area / 4.0
    return out


def closed_one_ring(nv: int, T: np.ndarray) -> np.ndarray:
    """Boolean adjacency with the diagonal: N[v] = {v} + neighbours of v."""
    A = np.eye(nv, dtype=bool)
    e = mesh_edges(T)
    A[e[:, 0], e[:, 1]] = True
    A[e[:, 1], e[:, 0]] = True
    return A


def nearest_indicators(d: np.ndarray, k: int) -> tuple[np.ndarray, np.ndarray]:
    """0/1 matrices of the k nearest pairs in each direction (ties to the lower index; only
    finite costs are ranked): cxy[m, n] = 1 iff n is among the k nearest Y vertices of m,
    cyx[m, n] = 1 iff m is among the k nearest X vertices of n."""
    nx, ny = d.shape
    fin = np.isfinite(d)
    dr = np.where(fin, d, np.inf)  # non-finite entries sort last and are dropped below
    cxy = np.zeros((nx, ny), dtype=np.float64)
    cyx = np.zeros((nx, ny), dtype=np.float64)
    rows = np.argsort(dr, axis=1, kind="stable")[:, : min(k, ny)]
    ri = np.broadcast_to(np.arange(nx)[:, None], rows.shape)
    cxy[ri, rows] = fin[ri, rows]
    cols = np.argsort(dr, axis=0, kind="stable")[: min(k, nx), :]
    ci = np.broadcast_to(np.arange(ny)[None, :], cols.shape)
    cyx[cols, ci] = fin[cols, ci]
    return cxy, cyx


def candidate_pairs(d: np.ndarray, k: int, TX: np.ndarray, TY: np.ndarray) -> np.ndarray:
    """Allowed vertex pairs for the top-k pruned product space.

    (m, n) is allowed iff n lies in the closed 1-ring of one of the k feature-nearest
    Y vertices of m, or m lies in the closed 1-ring of one of the k feature-nearest X
    vertices of n (ties to the lower index). Only finite costs are ranked: a row (or
    column) with fewer than k finite entries contributes just those."""
    nx, ny = d.shape
    cxy, cyx = nearest_indicators(d, k)
    # the products below count ring hits, exact in float64
    AX = closed_one_ring(nx, TX).astype(np.float64)
    AY = closed_one_ring(ny, TY).astype(np.float64)
    return ((cxy @ AY) > 0) | ((AX @ cyx) > 0)


@dataclass
class Problem:
    """ILP (P): min c^T x, A x = b, x binary.  Variables are product triangles."""

    nvx: int
    nvy: int
    vm: np.ndarray  # (P, 3) X vertex of each corner
    vn: np.ndarray  # (P, 3) Y vertex of each corner
    vtype: np.ndarray  # (P,)
    vx: np.ndarray  # X element index (triangle / edge / vertex by type)
    vy: np.ndarray  # Y element index
    vpat: np.ndarray  # rotation (tri-tri) or edge pattern
    cost: np.ndarray  # (P,) FP64 in [0, 1]
    row_ptr: np.ndarray
    row_var: np.ndarray
    row_coef: np.ndarray
    rhs: np.ndarray
    n_closed: int
    n_projx: int
    n_projy: int
    row_key: np.ndarray  # closedness: packed product-edge key; projection rows: -1

    @property
    def nvars(self) -> int:
        return int(self.vm.shape[0])

    @property
    def nrows(self) -> int:
        return int(self.rhs.shape[0])

    def row(self, r: int) -> tuple[np.ndarray, np.ndarray, int]:
        a, b = self.row_ptr[r], self.row_ptr[r + 1]
        return self.row_var[a:b], self.row_coef[a:b], int(self.rhs[r])

    def residual(self, x: np.ndarray) -> np.ndarray:
        """A x - b per row, exact integer arithmetic."""
        x = np.asarray(x, dtype=np.int64)
        prod = self.row_coef.astype(np.int64) * x[self.row_var]
        s = np.add.reduceat(prod, self.row_ptr[:-1]) if len(prod) else np.zeros(0, np.int64)
        empty = self.row_ptr[1:] == self.row_ptr[:-1]
        s = np.where(empty, 0, s)
        return s - self.rhs


def enumerate_product_space(TX: np.ndarray, TY: np.ndarray, allowed: np.ndarray):
    """All matching elements whose three vertex pairs are allowed, in canonical order."""
    TX = np.asarray(TX, dtype=np.int64)
    TY = np.asarray(TY, dtype=np.int64)
    EX, EY = mesh_edges(TX), mesh_edges(TY)
    nvx, nvy = allowed.shape
    out_m, out_n, out_t, out_x, out_y, out_p = [], [], [], [], [], []

    def emit(m, n, typ, x, y, p):
        out_m.append(m)
        out_n.append(n)
        out_t.append(np.full(len(x), typ, np.int64))
        out_x.append(x)
        out_y.append(y)
        out_p.append(p)

    # type 0: X triangle t, Y triangle s, cyclic rotation r: corner v pairs (t_v, s_{(v+r)%3})
    for t in range(len(TX)):
        m = TX[t]
        ok = np.stack([allowed[m[0], TY[:, r % 3]] & allowed[m[1], TY[:, (1 + r) % 3]] & allowed[m[2], TY[:, (2 + r) % 3]]
                       for r in range(3)], axis=1)  # (nTY, 3), row-major = (s, r)
        s, r = np.nonzero(ok)
        if len(s):
            n = np.stack([TY[s, (r + v) % 3] for v in range(3)], axis=1)
            emit(np.tile(m, (len(s), 1)), n, TT, np.full(len(s), t), s, r)
    # type 1: X triangle t, Y edge e, pattern p
    for t in range(len(TX)):
        m = TX[t]
        seqs = EY[:, None, :].repeat(6, 1)  # (E, 6, 2)
        n = np.take_along_axis(seqs, EDGE_PATTERNS[None, :, :].repeat(len(EY), 0), axis=2)  # (E, 6, 3)
        ok = allowed[m[0], n[:, :, 0]] & allowed[m[1], n[:, :, 1]] & allowed[m[2], n[:, :, 2]]
        e, p = np.nonzero(ok)
        if len(e):
            emit(np.tile(m, (len(e), 1)), n[e, p], XT_YE, np.full(len(e), t), e, p)
    # type 2: X edge e, Y triangle s, pattern p
    for e in range(len(EX)):
        mseq = EX[e][EDGE_PATTERNS]  # (6, 3)
        ok = np.stack([allowed[mseq[p, 0], TY[:, 0]] & allowed[mseq[p, 1], TY[:, 1]] & allowed[mseq[p, 2], TY[:, 2]]
                       for p in range(6)], axis=1)  # (nTY, 6) = (s, p)
        s, p = np.nonzero(ok)
        if len(s):
            emit(mseq[p], TY[s], XE_YT, np.full(len(s), e), s, p)
    # type 3: X triangle t, Y vertex n
    for t in range(len(TX)):
        m = TX[t]
        ok = allowed[m[0]] & allowed[m[1]] & allowed[m[2]]
        n = np.nonzero(ok)[0]
        if len(n):
            emit(np.tile(m, (len(n), 1)), np.stack([n, n, n], 1), XT_YV, np.full(len(n), t), n, np.zeros(len(n), np.int64))
    # type 4: X vertex m, Y triangle s
    for mv in range(nvx):
        ok = allowed[mv, TY[:, 0]] & allowed[mv, TY[:, 1]] & allowed[mv, TY[:, 2]]
        s = np.nonzero(ok)[0]
        if len(s):
            emit(np.full((len(s), 3), mv), TY[s], XV_YT, np.full(len(s), mv), s, np.zeros(len(s), np.int64))

    cat = lambda L, shape: np.concatenate(L) if L else np.zeros(shape, np.int64)  # noqa: E731
    return (cat(out_m, (0, 3)), cat(out_n, (0, 3)), cat(out_t, (0,)), cat(out_x, (0,)), cat(out_y, (0,)),
            cat(out_p, (0,)))


def build_problem(TX: np.ndarray, TY: np.ndarray, d: np.ndarray, allowed: np.ndarray | None = None,
                  cost_model: int = 0, VX: np.ndarray | None = None, VY: np.ndarray | None = None,
                  normalize: bool = True) -> Problem:
    """Product space, costs and constraint rows (closedness, then X projection, then Y projection).

    cost_model 0: c_p = mean of the three pair costs d; 1 (Eq. 2): c_p = sum over the three
    corners of (A_X(m_v) + A_Y(n_v)) d(m_v, n_v), A the mixed vertex areas of the meshes
    with positions VX, VY. Costs are then divided by the largest one unless normalize is off."""
    nvx, nvy = d.shape
    if allowed is None:
        allowed = np.ones((nvx, nvy), dtype=bool)
    TX = np.asarray(TX, dtype=np.int64)
    TY = np.asarray(TY, dtype=np.int64)
    vm, vn, vt, vx, vy, vp = enumerate_product_space(TX, TY, allowed)
    P = len(vt)
    # cost: mean of the three pair distances (or Eq. 2), normalised by the largest kept cost
    if cost_model == 1:
        aX = mixed_areas(VX, TX)
        aY = mixed_areas(VY, TY)
        c = sum((aX[vm[:, v]] + aY[vn[:, v]]) * d[vm[:, v], vn[:, v]] for v in range(3))
    else:
        c = (d[vm[:, 0], vn[:, 0]] + d[vm[:, 1], vn[:, 1]] + d[vm[:, 2], vn[:, 2]]) / 3.0
    cmax = c.max() if P else 1.0
    if normalize:
        c = c / cmax if cmax > 0 else c

    # closedness rows: each element's three boundary edges p_v -> p_{v+1}
    key = vm * nvy + vn  # product-vertex key, lexicographic in (m, n)
    a = key
    b = key[:, [1, 2, 0]]
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    coef = np.where(a < b, 1, -1)
    K = nvx * nvy
    ekey = (lo * K + hi).ravel()
    evar = np.repeat(np.arange(P), 3)
    ecoef = coef.ravel()
    order = np.lexsort((evar, ekey))
    ekey, evar, ecoef = ekey[order], evar[order], ecoef[order]
    ukeys, starts = np.unique(ekey, return_index=True)
    closed_ptr = np.append(starts, len(ekey))

    # projection rows: elements whose X side (resp. Y side) is the non-degenerate triangle
    xtri = np.where(np.isin(vt, [TT, XT_YE, XT_YV]), vx, -1)
    ytri = np.where(np.isin(vt, [TT, XE_YT, XV_YT]), vy, -1)
    rows_var = [evar]
    rows_coef = [ecoef]
    ptr = list(closed_ptr)
    rhs = [np.zeros(len(ukeys), np.int64)]
    off = len(ekey)
    for side, ntri in ((xtri, len(TX)), (ytri, len(TY))):
        sel = np.nonzero(side >= 0)[0]
        o = np.lexsort((sel, side[sel]))
        sel = sel[o]
        counts = np.bincount(side[sel], minlength=ntri)
        rows_var.append(sel)
        rows_coef.append(np.ones(len(sel), np.int64))
        cs = np.cumsum(counts)
        ptr += list(off + cs)
        off += len(sel)
        rhs.append(np.ones(ntri, np.int64))
    row_key = np.concatenate([ukeys, -np.ones(len(TX) + len(TY), np.int64)])
    return Problem(nvx, nvy, vm, vn, vt, vx, vy, vp, c,
                   np.array(ptr, np.int64), np.concatenate(rows_var).astype(np.int64),
                   np.concatenate(rows_coef).astype(np.int64), np.concatenate(rhs).astype(np.int64),
                   len(ukeys), len(TX), len(TY), row_key)


class Infeasible(Exception):
    pass


def gac(prob: Problem, fixed: np.ndarray) -> np.ndarray:
    """Generalised arc consistency of all rows, to a fixpoint.

    ``fixed``: int8 per variable, -1 free, 0/1 fixed. For a row sum_i a_i x_i = b with
    a_i in {+1, -1}, a free variable can take value v iff the remaining free variables
    can still reach the residual right-hand side. Raises Infeasible when some row has
    no solution."""
    fixed = fixed.copy()
    rv, rc, ptr = prob.row_var, prob.row_coef, prob.row_ptr
    nrow = prob.nrows
    row_of = np.repeat(np.arange(nrow), np.diff(ptr))
    while True:
        fv = fixed[rv]
        free = fv < 0
        val = np.where(free, 0, fv).astype(np.int64)
        s_fixed = np.bincount(row_of, weights=rc * val, minlength=nrow).astype(np.int64)
        npos = np.bincount(row_of, weights=(free & (rc > 0)), minlength=nrow).astype(np.int64)
        nneg = np.bincount(row_of, weights=(free & (rc < 0)), minlength=nrow).astype(np.int64)
        r = prob.rhs - s_fixed  # residual right-hand side for the free part
        if np.any(r > npos) or np.any(r < -nneg):
            raise Infeasible("row without solution")
        # support of value 1 / 0 for each free entry, by removing it from the free part
        rr = r[row_of]
        P_ = npos[row_of] - (rc > 0)
        Q_ = nneg[row_of] - (rc < 0)
        can1 = (rr - rc >= -Q_) & (rr - rc <= P_)
        can0 = (rr >= -Q_) & (rr <= P_)
        force0 = free & ~can1
        force1 = free & ~can0
        if np.any(force0 & force1):
            raise Infeasible("variable without support")
        if not (force0.any() or force1.any()):
            return fixed
        v0 = np.unique(rv[force0])
        v1 = np.unique(rv[force1])
        if np.intersect1d(v0, v1).size:
            raise Infeasible("conflicting forcings")
        fixed[v0] = 0
        fixed[v1] = 1


def presolve(prob: Problem) -> tuple[np.ndarray, float]:
    """Fix every variable that some row forces (GAC fixpoint). Returns (fixed, constant)."""
    fixed = gac(prob, -np.ones(prob.nvars, np.int8))
    const = float(prob.cost[fixed == 1].sum())
    return fixed, const


def make_problem(inst, topk="inst") -> tuple[Problem, np.ndarray, np.ndarray]:
    """Problem for a synthetic instance. Returns (problem, d, allowed)."""
    d = pair_distance(inst.FX, inst.FY)
    k = inst.topk if topk == "inst" else topk
    if k is None:
        allowed = np.ones(d.shape, dtype=bool)
    else:
        allowed = candidate_pairs(d, k, inst.X.T, inst.Y.T)
    return build_problem(inst.X.T, inst.Y.T, d, allowed), d, allowed


def point_map(prob: Problem, x: np.ndarray) -> np.ndarray:
    """Vertex pairs (m, n), sorted, at the corners of the elements set in x (the point-wise
    correspondence of a triangle matching)."""
    sel = np.asarray(x).astype(bool)
    pairs = np.stack([prob.vm[sel].ravel(), prob.vn[sel].ravel()], axis=1)
    return np.unique(pairs, axis=0) if len(pairs) else np.zeros((0, 2), np.int64)


def coarse_to_fine_candidates(pairs: np.ndarray, c2f_x: np.ndarray, c2f_y: np.ndarray, rings: int,
                              TX: np.ndarray, nvx: int, TY: np.ndarray, nvy: int) -> np.ndarray:
    """Fine pairs (m', n') with m' within `rings` edges of c2f_x[m] and n' within `rings` edges
    of c2f_y[n] for some coarse pair (m, n) (Sec. 4, coarse-to-fine). Boolean matrix powers of
    the closed 1-ring adjacency give the within-r relation."""
    def within(nv, T):
        A = closed_one_ring(nv, T).astype(np.float64)
        R = np.eye(nv)
        for _ in range(rings):
            R = ((R @ A) > 0).astype(np.float64)
        return R

    RX = within(nvx, TX)
    RY = within(nvy, TY)
    S = np.zeros((nvx, nvy))
    for m, n in np.asarray(pairs).reshape(-1, 2):
        S[c2f_x[m], c2f_y[n]] = 1.0
    return (RX.T @ S @ RY) > 0

