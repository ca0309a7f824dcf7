"""Structured parent grid of the unit cell for the full-order training solves on the device
(rom_fe_train): Q4 (2D) or hex8 (3D) elements with 2 x 2 (x 2) Gauss points, the periodic
fluctuation field (nodes on opposite faces identified), void elements removed (their nodes
carry no unknowns unless a kept element uses them), one node fixed against rigid translation
(Sec. 2.1: the fluctuation space V^p of the parent domain).

Numbering: cells with x fastest; the corner order of an element is counter-clockwise in the
(x, y) plane, then the same square at z + h; node id = sum_c idx_c N^c; dofs node by node over
the used nodes (the fixed one, the first corner of the first kept element, skipped),
component-minor."""
import itertools

import numpy as np

VOID = -1


def _corners(d):
    square = [(0, 0), (1, 0), (1, 1), (0, 1)]
    if d == 2:
        return square
    return [c + (0,) for c in square] + [c + (1,) for c in square]


class Grid:
    """Element arrays of an N^d grid on [0, 1]^d; phase_of(centroid) -> -1 (void), 0, 1, ..."""

    def __init__(self, d, N, phase_of):
        self.d, self.N = d, N
        h = 1.0 / N
        corners = np.array(_corners(d), dtype=float)
        self.nen = len(corners)
        ref = 2.0 * corners - 1.0                                    # reference coordinates of the nodes
        g = 1.0 / np.sqrt(3.0)
        gauss = np.array(list(itertools.product((-g, g), repeat=d)))
        self.ngp = len(gauss)
        # trilinear (bilinear) shape functions and their X^p gradients at the Gauss points
        lin = (1.0 + gauss[:, None, :] * ref[None, :, :]) / 2.0       # [ngp, nen, d] factors
        self.Nv = np.prod(lin, axis=2)
        self.dN = np.zeros((self.ngp, self.nen, d))
        for r in range(d):
            others = np.prod(np.delete(lin, r, axis=2), axis=2)
            self.dN[:, :, r] = (ref[None, :, r] / 2.0) * others * (2.0 / h)
        self.gw = np.full(self.ngp, (h / 2.0) ** d)
        cells = np.array(list(itertools.product(range(N), repeat=d)))[:, ::-1]
        phase = np.array([phase_of((c + 0.5) * h) for c in cells])
        keep = phase != VOID
        self.cells = cells[keep]
        self.el_phase = phase[keep].astype(np.int32)
        self.ne = len(self.cells)
        strides = N ** np.arange(d)
        conn = np.stack([(((self.cells + c.astype(int)) % N) * strides).sum(1) for c in corners], axis=1)
        self.conn = conn
        used = np.zeros(N ** d, bool)
        used[conn.ravel()] = True
        fixed = int(conn[0, 0])
        dof = -np.ones((N ** d, d), np.int64)
        nodes = [k for k in np.nonzero(used)[0] if k != fixed]
        dof[nodes] = np.arange(len(nodes) * d).reshape(-1, d)
        self.dof = dof
        self.ndof = len(nodes) * d
        self.edof = dof[conn].reshape(self.ne, self.nen * d).astype(np.int32)
        xnode = np.stack([(self.cells + c) * h for c in corners], axis=1)        # [ne, nen, d]
        self.X = np.einsum("ga,ead->egd", self.Nv, xnode)                          # Gauss points
        self.nq = self.ne * self.ngp
