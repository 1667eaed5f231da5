"""Seeded synthetic shape-matching instances.

Each instance is a pair of meshes X, Y (Y a deformed, relabelled copy of X),
per-vertex FP32 features F_X, F_Y (Y's = X's permuted by the relabelling plus
Gaussian noise), the ground-truth vertex map and the candidate rule
parameters. They stand in for the paper's learned URSSM features on FAUST_r /
SMAL / DT4D-H pairs (Sec. 4), which are not available here.

Nothing in this module computes any part of the matching method: costs,
candidates, product space, constraints and the solver are implemented twice,
independently, by ``oracle/`` and by the CUDA path, from these raw arrays.

Workloads (seed = config index XOR pair index):

* ``config1``  icosahedron vs relabelled copy + N(0, 0.01^2) vertex noise,
  16-d features, noise 0.05, full product space, 200 dual iterations.
* ``config2``  icosphere subdivision 2 (162 V / 320 T), smooth radial
  spherical-harmonic deformation (8 terms, degree <= 4, amplitude 0.1),
  relabelled, 64-d features, noise 0.05, top-k = 10, 500 iterations.
* ``config3``  icosphere subdivision 4 (2562 V / 5120 T), same deformation,
  128-d features, top-k = 16, run to a converged bound.
* ``config4``  64 uneven pairs (icospheres 80/320/1280 T, tori 96..1536 T),
  64-d features, top-k ~ U{8..24}, 300 iterations each.
* ``tet``      tetrahedron vs relabelled copy (exhaustive-search size).
* ``symmetric_pair(s)``  icosphere (subdivision s) vs a deformed, relabelled copy, with
  16-d features that are random combinations of the even-order real spherical
  harmonics of degree 1..4 at the vertex directions (plus noise 0.05 on Y). They
  are invariant under the half-turn about the z axis, which maps the icosphere onto
  itself, so two orientation-preserving matchings are equally good and the LP
  relaxation is not tight: the dual needs hundreds of iterations (s = 3: about 720
  to a change below 1e-6 over 20). A stand-in for the paper's slowly converging real
  shape pairs (intrinsic symmetries, ambiguous learned features).
* ``bipyramid_pair(n)``  bipyramid over an n-gon vs relabelled copy, 16-d
  features, noise 0.05, full product space: high-valence apexes give BDD layers
  wider than 8 (n = 12: up to 14, n = 16: up to 18).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import meshes as M


@dataclass
class Instance:
    name: str
    X: M.Mesh
    Y: M.Mesh
    FX: np.ndarray  # (nvX, D) float32
    FY: np.ndarray  # (nvY, D) float32
    perm: np.ndarray  # ground truth: X vertex v <-> Y vertex perm[v]
    topk: int | None  # None = full product space
    iters: int | None  # None = run until converged
    meta: dict = field(default_factory=dict)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def make_pair(X: M.Mesh, rng: np.random.Generator, dim: int, feat_noise: float,
              vertex_noise: float = 0.0, deform: bool = False) -> tuple[M.Mesh, np.ndarray, np.ndarray, np.ndarray]:
    Y0 = M.deform_radial(X, rng) if deform else X.copy()
    if vertex_noise > 0:
        Y0 = M.Mesh((Y0.V + vertex_noise * rng.standard_normal(Y0.V.shape)).astype(np.float32), Y0.T)
    Y, perm = M.relabel(Y0, rng)
    FX = rng.standard_normal((X.nv, dim)).astype(np.float32)
    FY = np.empty_like(FX)
    FY[perm] = FX + (feat_noise * rng.standard_normal(FX.shape)).astype(np.float32)
    return Y, FX, FY, perm


def tet(seed: int = 0, feat_noise: float = 0.05, dim: int = 16) -> Instance:
    rng = _rng(1000 + seed)
    X = M.tetrahedron()
    Y, FX, FY, perm = make_pair(X, rng, dim, feat_noise)
    return Instance("tet", X, Y, FX, FY, perm, None, 200)


def config1(pair: int = 0) -> Instance:
    rng = _rng(1 ^ pair)
    X = M.icosahedron()
    Y, FX, FY, perm = make_pair(X, rng, 16, 0.05, vertex_noise=0.01)
    return Instance("icosahedron-20T-full", X, Y, FX, FY, perm, None, 200)


def config2(pair: int = 0) -> Instance:
    rng = _rng(2 ^ pair)
    X = M.icosphere(2)
    Y, FX, FY, perm = make_pair(X, rng, 64, 0.05, deform=True)
    return Instance("icosphere2-320T-top10", X, Y, FX, FY, perm, 10, 500)


def config3(pair: int = 0) -> Instance:
    rng = _rng(3 ^ pair)
    X = M.icosphere(4)
    Y, FX, FY, perm = make_pair(X, rng, 128, 0.05, deform=True)
    return Instance("icosphere4-5120T-top16", X, Y, FX, FY, perm, 16, None)


def icosphere_pair(subdiv: int, dim: int, topk: int | None, seed: int, iters: int | None = None) -> Instance:
    """A generic deformed/relabelled icosphere pair (used for scaled variants)."""
    rng = _rng(seed)
    X = M.icosphere(subdiv)
    Y, FX, FY, perm = make_pair(X, rng, dim, 0.05, deform=True)
    return Instance(f"icosphere{subdiv}-{X.nt}T-top{topk}", X, Y, FX, FY, perm, topk, iters)


def symmetric_pair(subdiv: int = 3, dim: int = 16, feat_noise: float = 0.05, degree: int = 4,
                   seed: int = 77) -> Instance:
    rng = _rng(seed)
    X = M.icosphere(subdiv)
    V = X.V.astype(np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    theta = np.arccos(np.clip(V[:, 2], -1.0, 1.0))
    phi = np.arctan2(V[:, 1], V[:, 0])
    basis = np.stack([M._real_sph_harm(l, m, theta, phi) for l in range(1, degree + 1)
                      for m in range(-l, l + 1) if m % 2 == 0], axis=1)
    basis /= basis.std(axis=0, keepdims=True)
    W = rng.standard_normal((basis.shape[1], dim)) / np.sqrt(basis.shape[1])
    FX = (basis @ W).astype(np.float32)
    Y0 = M.deform_radial(X, rng)
    Y, perm = M.relabel(Y0, rng)
    FY = np.empty_like(FX)
    FY[perm] = FX + (feat_noise * rng.standard_normal(FX.shape)).astype(np.float32)
    return Instance(f"icosphere{subdiv}-{X.nt}T-halfturn-symmetric-top16", X, Y, FX, FY, perm, 16, None)


def bipyramid_pair(n: int, seed: int = 11) -> Instance:
    rng = _rng(seed ^ n)
    X = M.bipyramid(n)
    Y, FX, FY, perm = make_pair(X, rng, 16, 0.05)
    return Instance(f"bipyramid{n}-{X.nt}T-full", X, Y, FX, FY, perm, None, None)


def config4(n_pairs: int = 64) -> list[Instance]:
    out = []
    for p in range(n_pairs):
        rng = _rng(4 ^ p)
        if rng.random() < 0.5:
            X = M.icosphere(int(rng.integers(1, 4)))
        else:
            # tori with 96..1536 triangles: 2*n*m in that range, n, m >= 4
            while True:
                n = int(rng.integers(4, 40))
                m = int(rng.integers(4, 40))
                if 96 <= 2 * n * m <= 1536:
                    break
            X = M.torus(n, m)
        Y, FX, FY, perm = make_pair(X, rng, 64, 0.05, deform=True)
        k = int(rng.integers(8, 25))
        out.append(Instance(f"batch{p}-{X.nt}T-top{k}", X, Y, FX, FY, perm, k, 300))
    return out


def config5(n_pairs: int = 8, subdiv: int = 3) -> list[Instance]:
    """Pairs for the differentiated solve: icosphere X (subdivision 3: 1280 triangles)
    against a deformed, relabelled copy; raw 128-d N(0, 1) features (Y: permuted + N(0,
    0.05^2)) that a learned map turns into costs; top-16 candidates; 50 iterations."""
    out = []
    for p in range(n_pairs):
        rng = _rng(5 ^ p)
        X = M.icosphere(subdiv)
        Y, FX, FY, perm = make_pair(X, rng, 128, 0.05, deform=True)
        out.append(Instance(f"diff{p}-{X.nt}T-top16", X, Y, FX, FY, perm, 16, 50))
    return out


def coarse_fine_pair(subdiv: int = 2, dim: int = 16, feat_noise: float = 0.05, seed: int = 6):
    """An icosphere pair at two resolutions for coarse-to-fine solving.

    The fine pair is X_f = icosphere(subdiv) against a deformed, relabelled copy Y_f. The
    coarse pair uses the vertices of icosphere(subdiv - 1), which are the first vertices of
    X_f, on both sides (Y_c relabelled again). Returns (coarse, fine, c2f_x, c2f_y) with
    c2f_* mapping coarse vertex ids to fine ones; features of a coarse vertex are those of its
    fine vertex."""
    rng = _rng(seed)
    Xf = M.icosphere(subdiv)
    Yf, FXf, FYf, perm = make_pair(Xf, rng, dim, feat_noise, deform=True)
    Xc0 = M.icosphere(subdiv - 1)
    nc = Xc0.nv
    q = rng.permutation(nc).astype(np.int64)  # coarse Y id of X vertex j
    c2f_x = np.arange(nc, dtype=np.int32)
    c2f_y = np.empty(nc, np.int32)
    c2f_y[q] = perm[:nc]
    VYc = np.empty((nc, 3), np.float32)
    VYc[q] = Yf.V[perm[:nc]]
    Yc = M.Mesh(VYc, q[Xc0.T.astype(np.int64)].astype(np.int32))
    Xc = M.Mesh(Xf.V[:nc].copy(), Xc0.T)
    FYc = np.empty((nc, dim), np.float32)
    FYc[q] = FYf[perm[:nc]]
    coarse = Instance(f"coarse-{Xc.nt}T", Xc, Yc, FXf[:nc].copy(), FYc, q, None, 100)
    fine = Instance(f"fine-{Xf.nt}T", Xf, Yf, FXf, FYf, perm, None, 100)
    return coarse, fine, c2f_x, c2f_y


def multilevel_pair(levels=(1, 2, 3), dim: int = 16, feat_noise: float = 0.05, seed: int = 7):
    """An icosphere pair at several resolutions (subdivision levels), each level's vertices a
    prefix of the next one's on X; Y is a deformed, relabelled copy at the finest level and
    every coarser Y keeps the finest labels' relative order through a per-level relabelling.
    Returns [(Instance, c2f_x, c2f_y)] from coarse to fine, c2f_* mapping the level's vertex ids
    to the next level's (None for the finest)."""
    rng = _rng(seed)
    Xf = M.icosphere(levels[-1])
    Yf, FXf, FYf, perm = make_pair(Xf, rng, dim, feat_noise, deform=True)
    out, prev = [], None
    for lv in levels:
        X0 = M.icosphere(lv)
        nc = X0.nv
        q = rng.permutation(nc).astype(np.int64) if lv != levels[-1] else None
        if q is None:  # finest level: the generated pair itself
            inst, yfine = Instance(f"level{lv}-{Xf.nt}T", Xf, Yf, FXf, FYf, perm, None, 100), np.arange(Xf.nv)
        else:
            VY = np.empty((nc, 3), np.float32)
            VY[q] = Yf.V[perm[:nc]]
            FY = np.empty((nc, dim), np.float32)
            FY[q] = FYf[perm[:nc]]
            inst = Instance(f"level{lv}-{X0.nt}T", M.Mesh(Xf.V[:nc].copy(), X0.T), M.Mesh(VY, q[X0.T.astype(np.int64)].astype(np.int32)),
                            FXf[:nc].copy(), FY, q, None, 100)
            yfine = np.empty(nc, np.int64)
            yfine[q] = perm[:nc]  # level Y id -> finest Y id
        out.append([inst, yfine])
    # maps to the next level: X ids are prefixes; Y ids through the finest labels
    res = []
    for i, (inst, yfine) in enumerate(out):
        if i + 1 == len(out):
            res.append((inst, None, None))
            continue
        nxt_inst, nxt_yfine = out[i + 1]
        inv = np.full(int(nxt_yfine.max()) + 1, -1, np.int64)
        inv[nxt_yfine] = np.arange(len(nxt_yfine))
        res.append((inst, np.arange(inst.X.nv, dtype=np.int32), inv[yfine].astype(np.int32)))
    return res


def mlp_params(seed: int = 5, sizes=(128, 256, 64)) -> list[np.ndarray]:
    """Seeded weights of the 2-layer feature MLP (W1, b1, W2, b2; N(0, 1/fan_in), zero bias)."""
    rng = _rng(1000 + seed)
    out = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        out.append((rng.standard_normal((b, a)) / np.sqrt(a)).astype(np.float32))
        out.append(np.zeros(b, np.float32))
    return out


CONFIGS = {"config1": config1, "config2": config2, "config3": config3, "tet": tet}
