"""Step-domain Q2-Q1 mesh generator (geometry and numbering only).

The benchmark domain of Section 5.1 is a symmetric step: an inlet channel
[-l, 0] x [-1/2, 1/2] joined to a main channel [0, L] x [-1, 1].  Dirichlet
conditions hold on the inflow x1 = -l (parabolic profile 1 - 4 x2^2, Section 5.1)
and on every wall; the outflow x1 = L carries the natural condition.

This module builds node coordinates, element connectivity, the Dirichlet set
and the steady inflow profile.  It holds no finite-element arithmetic: the
oracle and the GPU path each integrate their own matrices from these arrays.

Conventions (an interface shared by both sides):
  * velocity (Q2) nodes sit on a grid of spacing h/2, where h is the element
    side; nodes are numbered column by column (x1 outer, x2 inner), which keeps
    the bandwidth of the scalar Q2 matrices near twice a column's node count;
  * a Q2 element lists its 9 nodes in the order a + 3 b, a, b in {0, 1, 2},
    a along x1 and b along x2;  its 4 pressure (Q1) vertices in the order
    a + 2 b, a, b in {0, 1};
  * pressure nodes are the element vertices, numbered column by column too.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    h: float                 # element side; velocity node spacing is h/2
    xy: np.ndarray           # (n_nodes, 2) velocity node coordinates
    elem_q2: np.ndarray      # (n_elem, 9) velocity node ids
    elem_q1: np.ndarray      # (n_elem, 4) pressure node ids
    pxy: np.ndarray          # (n_pnodes, 2) pressure node coordinates
    dirichlet: np.ndarray    # (n_nodes,) bool
    inflow: np.ndarray       # (n_nodes,) steady x1-velocity prescribed at Dirichlet nodes
    kind: str = "step"
    params: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return self.xy.shape[0]

    @property
    def n_elem(self) -> int:
        return self.elem_q2.shape[0]

    @property
    def n_pnodes(self) -> int:
        return self.pxy.shape[0]

    @property
    def free(self) -> np.ndarray:
        """Free (non-Dirichlet) velocity nodes, ascending."""
        return np.flatnonzero(~self.dirichlet).astype(np.int64)

    @property
    def dnodes(self) -> np.ndarray:
        """Dirichlet velocity nodes, ascending."""
        return np.flatnonzero(self.dirichlet).astype(np.int64)

    @property
    def n_v(self) -> int:
        """Free scalar velocity nodes; the paper's n_u is 2 n_v."""
        return int((~self.dirichlet).sum())


def _build(h, rects, classify, kind, params):
    """Generic builder over a union of axis-aligned rectangles.

    rects: list of (I0, I1, J0, J1) in units of the node spacing h/2 (inclusive
    node ranges; element corners at even offsets).  classify(I, J) returns
    (is_dirichlet, inflow_value) for a boundary node given integer coords.
    """
    hv = h / 2.0
    nodes = set()
    for (I0, I1, J0, J1) in rects:
        for I in range(I0, I1 + 1):
            for J in range(J0, J1 + 1):
                nodes.add((I, J))
    order = sorted(nodes)                       # column-major: I outer, J inner
    nid = {ij: k for k, ij in enumerate(order)}
    xy = np.array([(I * hv, J * hv) for (I, J) in order], dtype=np.float64)

    pnodes = sorted((I, J) for (I, J) in order if I % 2 == 0 and J % 2 == 0)
    pid = {ij: k for k, ij in enumerate(pnodes)}
    pxy = np.array([(I * hv, J * hv) for (I, J) in pnodes], dtype=np.float64)

    cells = set()
    for (I0, I1, J0, J1) in rects:
        for I in range(I0, I1, 2):
            for J in range(J0, J1, 2):
                cells.add((I, J))
    cells = sorted(cells)
    e2 = np.empty((len(cells), 9), dtype=np.int64)
    e1 = np.empty((len(cells), 4), dtype=np.int64)
    for e, (I, J) in enumerate(cells):
        for b in range(3):
            for a in range(3):
                e2[e, a + 3 * b] = nid[(I + a, J + b)]
        for b in range(2):
            for a in range(2):
                e1[e, a + 2 * b] = pid[(I + 2 * a, J + 2 * b)]

    dirichlet = np.zeros(len(order), dtype=bool)
    inflow = np.zeros(len(order), dtype=np.float64)
    for k, (I, J) in enumerate(order):
        d, val = classify(I, J)
        dirichlet[k] = d
        inflow[k] = val
    return Mesh(h=h, xy=xy, elem_q2=e2, elem_q1=e1, pxy=pxy, dirichlet=dirichlet,
                inflow=inflow, kind=kind, params=params)


def _units(v, hv):
    q = v / hv
    n = int(round(q))
    if abs(q - n) > 1e-9:
        raise ValueError(f"length {v} is not a multiple of the node spacing {hv}")
    return n


def step_mesh(h: float, L: float = 5.0, inlet_len: float = 1.0) -> Mesh:
    """Symmetric step of Section 5.1: inlet [-inlet_len,0]x[-1/2,1/2], main [0,L]x[-1,1]."""
    hv = h / 2.0
    nl, nL = _units(inlet_len, hv), _units(L, hv)
    nh, n1 = _units(0.5, hv), _units(1.0, hv)
    if nh % 2 or nl % 2 or nL % 2:
        raise ValueError("element side must divide 1/2, the inlet length and L")
    rects = [(-nl, 0, -nh, nh), (0, nL, -n1, n1)]

    def classify(I, J):
        y = J * hv
        if I == -nl and abs(J) <= nh:                      # inflow x1 = -l
            return True, 1.0 - 4.0 * y * y
        if abs(J) == nh and -nl <= I <= 0:                 # inlet walls
            return True, 0.0
        if I == 0 and nh <= abs(J) <= n1:                  # step faces
            return True, 0.0
        if abs(J) == n1 and 0 <= I <= nL:                  # main walls (incl. outflow corners)
            return True, 0.0
        return False, 0.0

    return _build(h, rects, classify, "step", dict(L=L, inlet_len=inlet_len))


def channel_mesh(h: float, L: float = 2.0) -> Mesh:
    """Straight channel [0,L]x[-1,1]: inflow 1 - x2^2 at x1 = 0, walls x2 = +-1, outflow x1 = L.

    Poiseuille flow is exactly representable here, which pins the assembly.
    """
    hv = h / 2.0
    nL, n1 = _units(L, hv), _units(1.0, hv)
    rects = [(0, nL, -n1, n1)]

    def classify(I, J):
        y = J * hv
        if I == 0:
            return True, 1.0 - y * y
        if abs(J) == n1:
            return True, 0.0
        return False, 0.0

    return _build(h, rects, classify, "channel", dict(L=L))
