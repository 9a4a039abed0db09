"""Embedding of the velocity nodes of a mesh in the regular lattice of its
bounding box (node spacing h/2), the grid on which the learned mean-Oseen solve
works.  Layout only: no solver arithmetic."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Lattice:
    nx: int                  # lattice points along x1
    ny: int                  # lattice points along x2
    ix: np.ndarray           # (n_nodes,) x1 lattice index of every velocity node
    iy: np.ndarray           # (n_nodes,) x2 lattice index
    mask: np.ndarray         # (ny, nx) 1.0 on lattice points that are mesh nodes
    free: np.ndarray         # free velocity node ids (the unknowns, in order)


def node_lattice(mesh) -> Lattice:
    """Lattice indices of the mesh's velocity nodes (exact: nodes sit at integer
    multiples of h/2)."""
    hv = mesh.h / 2.0
    lo = mesh.xy.min(axis=0)
    ij = np.rint((mesh.xy - lo) / hv).astype(np.int64)
    nx, ny = int(ij[:, 0].max()) + 1, int(ij[:, 1].max()) + 1
    mask = np.zeros((ny, nx))
    mask[ij[:, 1], ij[:, 0]] = 1.0
    return Lattice(nx=nx, ny=ny, ix=ij[:, 0], iy=ij[:, 1], mask=mask, free=mesh.free)


def scatter_nodes(lat: Lattice, values: np.ndarray) -> np.ndarray:
    """(n_nodes,) node values -> (ny, nx) lattice image, zero off the mesh."""
    img = np.zeros((lat.ny, lat.nx))
    img[lat.iy, lat.ix] = values
    return img


def gather_nodes(lat: Lattice, img: np.ndarray) -> np.ndarray:
    """(ny, nx) lattice image -> (n_nodes,) node values."""
    return img[lat.iy, lat.ix]


def gaussian_residuals(n_free: int, count: int, seed: int = 1234) -> np.ndarray:
    """Seeded standard normal draws on the free velocity unknowns of both
    components: (count, 2 n_free)."""
    return np.random.default_rng(seed).standard_normal((count, 2 * n_free))


def he_normal_params(channels: int, depth: int, seed: int = 0, c_in: int = 5, c_out: int = 2) -> np.ndarray:
    """Seeded initial weights of the learned solve's network, flat float32 in the
    library's layout (per layer W[out][in][3][3] then b[out]): He-normal weights
    (std sqrt(2 / fan_in)), zero biases, the last layer scaled by 0.1 so the
    untrained network starts near zero output."""
    rng = np.random.default_rng(seed)
    sizes = [c_in] + [channels] * (depth - 1) + [c_out]
    out = []
    for k in range(depth):
        W = rng.standard_normal((sizes[k + 1], sizes[k], 3, 3)) * np.sqrt(2.0 / (sizes[k] * 9))
        if k == depth - 1:
            W *= 0.1
        out += [W.ravel(), np.zeros(sizes[k + 1])]
    return np.concatenate(out).astype(np.float32)
