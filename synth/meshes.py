"""Seeded synthetic triangle meshes.

Closed, consistently oriented (counter-clockwise seen from outside) triangle
meshes that stand in for the paper's shape datasets (FAUST_r, SMAL, DT4D-H at
about 450 faces, Sec. 4 "Datasets"), which are not available here:

* ``tetrahedron``   4 vertices,    4 triangles (exhaustive-search size)
* ``icosahedron``  12 vertices,   20 triangles
* ``icosphere(s)`` 10*4^s+2 vertices, 20*4^s triangles (s = 2: 162 / 320,
  s = 4: 2562 / 5120)
* ``torus(n, m)``  n*m vertices, 2*n*m triangles (genus 1)
* ``bipyramid(n)`` n+2 vertices, 2*n triangles: two apexes of valence n over an
  n-gon, so the constraint rows around the apexes are long and their BDDs wide

This module holds only geometry generation (no part of the matching method)
and is shared by the oracle and the CUDA path as the single source of inputs.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    V: np.ndarray  # (nv, 3) float32 vertex positions
    T: np.ndarray  # (nt, 3) int32 triangles, counter-clockwise

    @property
    def nv(self) -> int:
        return int(self.V.shape[0])

    @property
    def nt(self) -> int:
        return int(self.T.shape[0])

    def copy(self) -> "Mesh":
        return Mesh(self.V.copy(), self.T.copy())


def _orient_outward(V: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Flip triangles of a star-shaped closed surface so normals point away from the centroid."""
    c = V.mean(axis=0)
    a, b, d = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    n = np.cross(b - a, d - a)
    out = np.einsum("ij,ij->i", n, (a + b + d) / 3.0 - c) > 0
    T = T.copy()
    T[~out] = T[~out][:, [0, 2, 1]]
    return T


def tetrahedron() -> Mesh:
    V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    T = np.array([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]], dtype=np.int64)
    return Mesh(V.astype(np.float32), _orient_outward(V, T).astype(np.int32))


def icosahedron() -> Mesh:
    p = (1.0 + 5.0 ** 0.5) / 2.0
    V = []
    for s1 in (-1, 1):
        for s2 in (-1, 1):
            V += [(0, s1, s2 * p), (s1, s2 * p, 0), (s2 * p, 0, s1)]
    V = np.array(V, dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    # faces = triples of mutually nearest neighbours (edge length is the minimum distance)
    D = np.linalg.norm(V[:, None] - V[None], axis=2)
    e = D[D > 1e-9].min()
    adj = np.abs(D - e) < 1e-6
    T = [
        (i, j, k)
        for i in range(12)
        for j in range(i + 1, 12)
        for k in range(j + 1, 12)
        if adj[i, j] and adj[j, k] and adj[i, k]
    ]
    T = np.array(T, dtype=np.int64)
    assert T.shape == (20, 3)
    return Mesh(V.astype(np.float32), _orient_outward(V, T).astype(np.int32))


def icosphere(subdiv: int) -> Mesh:
    """Loop-style 1-to-4 midpoint subdivision of the icosahedron, projected to the unit sphere."""
    m = icosahedron()
    V = [tuple(v) for v in m.V.astype(np.float64)]
    T = m.T.astype(np.int64)
    for _ in range(subdiv):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                p = (np.asarray(V[a]) + np.asarray(V[b])) / 2.0
                p /= np.linalg.norm(p)
                cache[key] = len(V)
                V.append(tuple(p))
            return cache[key]

        nT = []
        for a, b, c in T:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nT += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        T = np.array(nT, dtype=np.int64)
    Va = np.array(V, dtype=np.float64)
    return Mesh(Va.astype(np.float32), T.astype(np.int32))


def torus(n: int, m: int, R: float = 1.0, r: float = 0.4) -> Mesh:
    """n x m grid on a torus (n around the major circle, m around the tube), 2nm triangles."""
    assert n >= 3 and m >= 3
    i, j = np.meshgrid(np.arange(n), np.arange(m), indexing="ij")
    u = 2 * np.pi * i / n
    v = 2 * np.pi * j / m
    V = np.stack([(R + r * np.cos(v)) * np.cos(u), (R + r * np.cos(v)) * np.sin(u), r * np.sin(v)], -1)
    V = V.reshape(-1, 3)
    idx = lambda a, b: (a % n) * m + (b % m)  # noqa: E731
    T = []
    for a in range(n):
        for b in range(m):
            p, q, s, t = idx(a, b), idx(a + 1, b), idx(a + 1, b + 1), idx(a, b + 1)
            T += [(p, q, s), (p, s, t)]
    return Mesh(V.astype(np.float32), np.array(T, dtype=np.int32))


def bipyramid(n: int) -> Mesh:
    """Two apexes (vertices n, n + 1) over a regular n-gon in the z = 0 plane."""
    assert n >= 3
    a = 2 * np.pi * np.arange(n) / n
    V = np.concatenate([np.stack([np.cos(a), np.sin(a), np.zeros(n)], 1), [[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]]])
    T = []
    for i in range(n):
        j = (i + 1) % n
        T += [(i, j, n), (j, i, n + 1)]
    T = np.array(T, dtype=np.int64)
    return Mesh(V.astype(np.float32), _orient_outward(V, T).astype(np.int32))


def _real_sph_harm(l: int, mm: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Unnormalised real spherical harmonic of degree l, order mm (|mm| <= l)."""
    from scipy.special import lpmv

    P = lpmv(abs(mm), l, np.cos(theta))
    if mm > 0:
        return P * np.cos(mm * phi)
    if mm < 0:
        return P * np.sin(-mm * phi)
    return P


def deform_radial(mesh: Mesh, rng: np.random.Generator, n_terms: int = 8, max_degree: int = 4,
                  amplitude: float = 0.1) -> Mesh:
    """Smooth radial displacement: sum of ``n_terms`` random real spherical harmonics of
    degree <= ``max_degree``, scaled so that the largest displacement is ``amplitude``."""
    V = mesh.V.astype(np.float64)
    c = V.mean(axis=0)
    d = V - c
    rad = np.linalg.norm(d, axis=1)
    theta = np.arccos(np.clip(d[:, 2] / np.maximum(rad, 1e-12), -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    f = np.zeros(len(V))
    for _ in range(n_terms):
        l = int(rng.integers(1, max_degree + 1))
        mm = int(rng.integers(-l, l + 1))
        f += rng.standard_normal() * _real_sph_harm(l, mm, theta, phi)
    s = np.abs(f).max()
    if s > 0:
        f *= amplitude / s
    V2 = c + d * (1.0 + f)[:, None]
    return Mesh(V2.astype(np.float32), mesh.T.copy())


def relabel(mesh: Mesh, rng: np.random.Generator, shuffle_faces: bool = True) -> tuple[Mesh, np.ndarray]:
    """Random vertex relabelling. Returns (Y, perm) with Y.V[perm[v]] == mesh.V[v].

    Faces are mapped through ``perm``; optionally their order is shuffled and each
    face's vertex order is rotated cyclically (orientation is preserved)."""
    nv = mesh.nv
    perm = rng.permutation(nv).astype(np.int64)
    V = np.empty_like(mesh.V)
    V[perm] = mesh.V
    T = perm[mesh.T.astype(np.int64)]
    if shuffle_faces:
        T = T[rng.permutation(len(T))]
        rot = rng.integers(0, 3, size=len(T))
        T = np.stack([T[np.arange(len(T)), (rot + k) % 3] for k in range(3)], axis=1)
    return Mesh(V, T.astype(np.int32)), perm
