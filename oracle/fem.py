"""Oracle of the robust finite-element update that consumes the block matches.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.

Plain numpy / scipy in FP64, following Sec. 3 of the paper ("Estimation of
brain deformation is based on the finite element analysis ..."): mesh vertex
displacements U balance the stiffness of a linear elastic model against the
block-matching displacements D,

    F_i = K U_i,    U_{i+1} = [K + H^T S H]^{-1} [H^T S D + F_i],

with K the stiffness matrix, H the interpolation from mesh vertices to the
block centres and S the diagonal confidence of the block matches; Sec. 5 lists
the number of approximation (outlier rejection) steps N_rej, the number of
interpolation steps N_int and the fraction F_r of blocks rejected as outliers.
The paper leaves the mesh, the material, S and the rejection rule to its
references; the readings taken here are:

* mesh: a structured grid of 8-node hexahedra whose vertices lie every g
  voxels from the origin (the last vertex on each axis at or past the
  volume's last voxel); a hexahedron is part of the model when the mask is
  set at the voxel at its centre (rounded down, clamped into the volume);
  vertices of no such element carry no unknowns (U = 0 there);
* material: homogeneous, isotropic linear elasticity with Young's modulus E
  and Poisson ratio nu, lengths in voxels; K_e by 2x2x2 Gauss quadrature;
* H: trilinear interpolation inside the element holding the block centre
  (the element of index floor(c / g), clamped to the grid);
* S: s_k = NCC_k for a valid match with positive NCC whose element is in the
  model, else 0;
* steps: U_0 = 0; N_rej approximation steps, each a solve followed by the
  rejection of n_rej = floor(0.5 + F_r * n) of the n blocks with s_k > 0
  (those with the largest squared residual |D_k - H_k U|^2, ties to the
  lower block index, never a block whose residual is at most R2_MIN =
  1e-6 voxel^2, i.e. a thousandth of a voxel: such a block agrees with the
  field and its rank would be set by rounding), which get s_k = 0;
  then N_int interpolation steps (solves without rejection); a step with
  no block left with s_k > 0 keeps U_{i+1} = U_i (the system is then K U =
  K U_i, whose solutions differ by rigid motions; U_i is the one with the
  least correction).

Every function names the step of the method it computes; the linear solve is
scipy's sparse direct solver (a library primitive).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ---- material and element (Sec. 3: K, the mechanical stiffness matrix) -----

def lame(E: float, nu: float):
    """Lame parameters (lambda, mu) of an isotropic material."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def elasticity_matrix(E: float, nu: float) -> np.ndarray:
    """6x6 stress-strain matrix, Voigt order (xx, yy, zz, xy, yz, zx), shear
    strains as engineering strains (gamma = 2 epsilon)."""
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    for i in range(3):
        D[i, i] = lam + 2.0 * mu
        D[3 + i, 3 + i] = mu
    return D


def local_node(a: int):
    """Corner offsets (ax, ay, az) in {0, 1} of local node a = ax + 2 ay + 4 az."""
    return a & 1, (a >> 1) & 1, (a >> 2) & 1


def element_stiffness(g: float, E: float, nu: float) -> np.ndarray:
    """24x24 stiffness of a cube element of edge g; dof 3 a + c is component c
    (x, y, z) of local node a.  Trilinear shape functions
    N_a = prod_i (1 + s_i xi_i) / 2 with s_i = +-1, integrated with 2x2x2
    Gauss points at xi = +-1/sqrt(3) (weights 1)."""
    D = elasticity_matrix(E, nu)
    q = 1.0 / math.sqrt(3.0)
    K = np.zeros((24, 24))
    detJ = (g / 2.0) ** 3
    for gx in (-q, q):
        for gy in (-q, q):
            for gz in (-q, q):
                xi = (gx, gy, gz)
                dN = np.zeros((8, 3))  # dN_a / dx_j
                for a in range(8):
                    s = [2 * o - 1 for o in local_node(a)]
                    f = [(1.0 + s[i] * xi[i]) / 2.0 for i in range(3)]
                    for j in range(3):
                        d = s[j] / 2.0
                        for i in range(3):
                            if i != j:
                                d *= f[i]
                        dN[a, j] = d * (2.0 / g)  # d xi / dx = 2 / g
                Bm = np.zeros((6, 24))
                for a in range(8):
                    dx, dy, dz = dN[a]
                    c = 3 * a
                    Bm[0, c + 0] = dx
                    Bm[1, c + 1] = dy
                    Bm[2, c + 2] = dz
                    Bm[3, c + 0] = dy
                    Bm[3, c + 1] = dx
                    Bm[4, c + 1] = dz
                    Bm[4, c + 2] = dy
                    Bm[5, c + 0] = dz
                    Bm[5, c + 2] = dx
                K += Bm.T @ D @ Bm * detJ
    return K


# ---- mesh -------------------------------------------------------------------

def grid_nodes(dims, g: int):
    """Vertices per axis (x, y, z) for a volume of dims (nx, ny, nz)."""
    return tuple((n - 1 + g - 1) // g + 1 for n in dims)


def active_elements(mask: np.ndarray, g: int) -> np.ndarray:
    """bool [Ez][Ey][Ex]: element (i, j, k) is in the model when the mask is
    set at its centre voxel (i g + g // 2, ...), clamped into the volume."""
    nz, ny, nx = mask.shape
    Nx, Ny, Nz = grid_nodes((nx, ny, nz), g)
    act = np.zeros((Nz - 1, Ny - 1, Nx - 1), dtype=bool)
    for k in range(Nz - 1):
        z = min(k * g + g // 2, nz - 1)
        for j in range(Ny - 1):
            y = min(j * g + g // 2, ny - 1)
            for i in range(Nx - 1):
                x = min(i * g + g // 2, nx - 1)
                act[k, j, i] = mask[z, y, x] != 0
    return act


def element_nodes(i: int, j: int, k: int, Nx: int, Ny: int):
    """Global vertex indices of element (i, j, k), in local node order."""
    out = []
    for a in range(8):
        ax, ay, az = local_node(a)
        out.append((i + ax) + Nx * ((j + ay) + Ny * (k + az)))
    return out


def assemble_stiffness(act: np.ndarray, g: int, E: float, nu: float, Nx: int, Ny: int, Nz: int):
    """Global K (3 n_vertices square, CSR) summed over the model's elements."""
    Ke = element_stiffness(g, E, nu)
    rows, cols, vals = [], [], []
    Ez, Ey, Ex = act.shape
    for k in range(Ez):
        for j in range(Ey):
            for i in range(Ex):
                if not act[k, j, i]:
                    continue
                nodes = element_nodes(i, j, k, Nx, Ny)
                dof = np.array([3 * n + c for n in nodes for c in range(3)])
                rows.append(np.repeat(dof, 24))
                cols.append(np.tile(dof, 24))
                vals.append(Ke.ravel())
    n = 3 * Nx * Ny * Nz
    if not rows:
        return sp.csr_matrix((n, n))
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()


def active_nodes(act: np.ndarray, Nx: int, Ny: int, Nz: int) -> np.ndarray:
    """bool [n_vertices]: vertices of at least one element of the model."""
    on = np.zeros(Nx * Ny * Nz, dtype=bool)
    Ez, Ey, Ex = act.shape
    for k in range(Ez):
        for j in range(Ey):
            for i in range(Ex):
                if act[k, j, i]:
                    on[element_nodes(i, j, k, Nx, Ny)] = True
    return on


# ---- interpolation H and confidence S ---------------------------------------

def block_cell(c, g: int, Nx: int, Ny: int, Nz: int):
    """Element (i, j, k) holding point c = (x, y, z) and the local
    coordinates t in [0, 1]^3 inside it."""
    cell, t = [], []
    for v, N in zip(c, (Nx, Ny, Nz)):
        i = min(max(int(v) // g, 0), N - 2)
        cell.append(i)
        t.append(v / g - i)
    return tuple(cell), tuple(t)


def trilinear_weights(t):
    """Weights of the 8 local nodes at local coordinates t."""
    w = np.empty(8)
    for a in range(8):
        ax, ay, az = local_node(a)
        w[a] = (t[0] if ax else 1.0 - t[0]) * (t[1] if ay else 1.0 - t[1]) * (t[2] if az else 1.0 - t[2])
    return w


def interpolation(centers: np.ndarray, act: np.ndarray, g: int, Nx: int, Ny: int, Nz: int):
    """H (3 n_blocks x 3 n_vertices, CSR) and the bool mask of the blocks
    whose element is in the model (the others' rows are zero)."""
    n = len(centers)
    rows, cols, vals = [], [], []
    inside = np.zeros(n, dtype=bool)
    for b in range(n):
        (i, j, k), t = block_cell(centers[b], g, Nx, Ny, Nz)
        if not act[k, j, i]:
            continue
        inside[b] = True
        w = trilinear_weights(t)
        for a, node in enumerate(element_nodes(i, j, k, Nx, Ny)):
            for c in range(3):
                rows.append(3 * b + c)
                cols.append(3 * node + c)
                vals.append(w[a])
    H = sp.coo_matrix((vals, (rows, cols)), shape=(3 * n, 3 * Nx * Ny * Nz)).tocsr()
    return H, inside


def confidence(ncc: np.ndarray, valid: np.ndarray, inside: np.ndarray) -> np.ndarray:
    """Diagonal of S: the peak NCC of a valid match with positive NCC whose
    element is in the model, else 0."""
    s = np.where((valid != 0) & inside & (ncc > 0), ncc, 0.0)
    return np.nan_to_num(s, nan=0.0)


# ---- rejection (Sec. 5: N_rej approximation steps, fraction F_r) -------------

R2_MIN = 1e-6  # squared residual (voxel^2) at or below which a block is never an outlier

def n_reject(n: int, fr: float) -> int:
    """Blocks rejected in one approximation step: floor(0.5 + F_r n), the
    rounding the paper uses for the selection count."""
    return int(math.floor(0.5 + n * fr))


def residuals(H, U: np.ndarray, disp: np.ndarray) -> np.ndarray:
    """Squared distance |D_k - H_k U|^2 of every block."""
    r = disp.reshape(-1).astype(np.float64) - H @ U
    r = r.reshape(-1, 3)
    return (r * r).sum(axis=1)


def reject(s: np.ndarray, r2: np.ndarray, fr: float) -> np.ndarray:
    """Indices of the blocks rejected in one approximation step: among the
    blocks with s > 0 and r2 > R2_MIN, the floor(0.5 + F_r n) largest r2 (n
    the count of s > 0), ties to the lower index."""
    cand = np.nonzero(s > 0)[0]
    k = min(n_reject(len(cand), fr), int((r2[cand] > R2_MIN).sum()))
    if k <= 0:
        return np.zeros(0, dtype=np.int64)
    order = sorted(cand.tolist(), key=lambda b: (-r2[b], b))
    return np.array(order[:k], dtype=np.int64)


# ---- the update (Sec. 3 equation) ---------------------------------------------

class Model:
    """Mesh, K and H of one registration (the parts that do not change
    between steps)."""

    def __init__(self, mask: np.ndarray, centers: np.ndarray, g: int, E: float, nu: float):
        nz, ny, nx = mask.shape
        self.g = g
        self.N = grid_nodes((nx, ny, nz), g)
        Nx, Ny, Nz = self.N
        self.act = active_elements(mask, g)
        self.K = assemble_stiffness(self.act, g, E, nu, Nx, Ny, Nz)
        self.node_on = active_nodes(self.act, Nx, Ny, Nz)
        self.dof_on = np.repeat(self.node_on, 3)
        self.H, self.inside = interpolation(np.asarray(centers), self.act, g, Nx, Ny, Nz)

    def step(self, U: np.ndarray, s: np.ndarray, disp: np.ndarray) -> np.ndarray:
        """U_{i+1} = [K + H^T S H]^{-1} [H^T S D + K U_i] over the model's
        unknowns (the other vertices stay at 0)."""
        if not (s > 0).any():
            # no trusted block: K U = K U_i, and U_i is the solution (the
            # correction of least norm), since K alone fixes no rigid motion
            return U.copy()
        S3 = sp.diags(np.repeat(s, 3))
        A = (self.K + self.H.T @ S3 @ self.H).tocsr()
        rhs = self.H.T @ (S3 @ disp.reshape(-1).astype(np.float64)) + self.K @ U
        on = np.nonzero(self.dof_on)[0]
        out = np.zeros_like(U)
        if len(on):
            out[on] = spla.spsolve(A[on][:, on].tocsc(), rhs[on])
        return out


def update(mask, centers, disp, ncc, valid, g: int, E: float, nu: float, n_rej: int, n_int: int, fr: float,
           model: Model | None = None):
    """The robust update: returns (U [n_vertices][3], s [n_blocks] after the
    rejections, rejected [n_blocks] bool, the step in which each block was
    rejected (-1: never))."""
    m = model or Model(mask, centers, g, E, nu)
    disp = np.asarray(disp, dtype=np.float64).reshape(-1, 3)
    s = confidence(np.asarray(ncc, dtype=np.float64), np.asarray(valid), m.inside)
    U = np.zeros(3 * len(m.node_on))
    when = np.full(len(s), -1, dtype=np.int64)
    for it in range(n_rej + n_int):
        U = m.step(U, s, disp)
        if it < n_rej:
            out = reject(s, residuals(m.H, U, disp), fr)
            s[out] = 0.0
            when[out] = it
    return U.reshape(-1, 3), s, when >= 0, when
