"""Pins of the finite-element oracle (oracle/fem.py) against what mechanics
and the update of Sec. 3 fix, independently of the oracle's own formulas:
rigid motions cost no energy, a uniform strain stores the closed-form energy
density, linear fields pass the patch test and are reproduced by trilinear
interpolation, a translation or an affine field sampled at the blocks is a
fixed point of the update, planted outliers are the ones rejected, and the
sparse assembly equals a dense one written with plain loops."""
import math

import numpy as np
import pytest

from oracle import fem

G, E, NU = 4, 2.0, 0.3


def _rigid_modes(g):
    """The six rigid motions of a cube of edge g (3 translations and 3
    infinitesimal rotations about its corner), as 24-vectors."""
    X = np.array([[g * o for o in fem.local_node(a)] for a in range(8)], dtype=float)
    modes = []
    for c in range(3):
        u = np.zeros((8, 3))
        u[:, c] = 1.0
        modes.append(u.ravel())
    for axis in range(3):
        w = np.zeros(3)
        w[axis] = 1.0
        modes.append(np.cross(w, X).ravel())
    return modes


def test_element_stiffness_symmetric_psd_with_six_rigid_modes():
    Ke = fem.element_stiffness(G, E, NU)
    assert np.allclose(Ke, Ke.T, atol=1e-14)
    ev = np.linalg.eigvalsh(Ke)
    assert ev.min() > -1e-12 * ev.max()
    assert (np.abs(ev) < 1e-10 * ev.max()).sum() == 6  # full integration: no hourglass modes
    for u in _rigid_modes(G):
        assert np.abs(Ke @ u).max() < 1e-12 * np.abs(Ke).max()


@pytest.mark.parametrize("g", [1, 3, 4])
def test_uniform_strain_energy_matches_closed_form(g):
    # a linear field is represented exactly, so 1/2 u^T K_e u is the energy
    # density times the volume g^3: uniaxial strain (lambda + 2 mu) eps^2 / 2,
    # simple shear mu gamma^2 / 2, volumetric (3 lambda + 2 mu) 3 eps^2 / 2
    Ke = fem.element_stiffness(g, E, NU)
    lam, mu = fem.lame(E, NU)
    X = np.array([[g * o for o in fem.local_node(a)] for a in range(8)], dtype=float)
    eps = 1e-2
    for comp in range(3):
        u = np.zeros((8, 3))
        u[:, comp] = eps * X[:, comp]
        en = 0.5 * u.ravel() @ Ke @ u.ravel()
        assert math.isclose(en, 0.5 * (lam + 2 * mu) * eps ** 2 * g ** 3, rel_tol=1e-12)
    for a_, b_ in ((0, 1), (1, 2), (2, 0)):
        u = np.zeros((8, 3))
        u[:, a_] = eps * X[:, b_]  # u_a = gamma x_b: engineering shear gamma
        en = 0.5 * u.ravel() @ Ke @ u.ravel()
        assert math.isclose(en, 0.5 * mu * eps ** 2 * g ** 3, rel_tol=1e-12)
    u = eps * X
    en = 0.5 * u.ravel() @ Ke @ u.ravel()
    assert math.isclose(en, 0.5 * (9 * lam + 6 * mu) * eps ** 2 * g ** 3, rel_tol=1e-12)


def test_lame_parameters_closed_form():
    lam, mu = fem.lame(1.0, 0.25)
    assert math.isclose(lam, 0.4) and math.isclose(mu, 0.4)
    D = fem.elasticity_matrix(1.0, 0.25)
    # uniaxial stress: strain (1, -nu, -nu) gives stress (E, 0, 0)
    s = D @ np.array([1.0, -0.25, -0.25, 0, 0, 0])
    assert np.allclose(s, [1.0, 0, 0, 0, 0, 0], atol=1e-15)


def _mask(nx, ny, nz, frac=0.45):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = ((x - (nx - 1) / 2) / (frac * nx)) ** 2 + ((y - (ny - 1) / 2) / (frac * ny)) ** 2 + \
        ((z - (nz - 1) / 2) / (frac * nz)) ** 2
    return (r <= 1.0).astype(np.uint8)


def test_patch_test_linear_field_no_interior_force():
    mask = np.ones((13, 13, 13), dtype=np.uint8)
    Nx, Ny, Nz = fem.grid_nodes((13, 13, 13), G)
    act = fem.active_elements(mask, G)
    assert act.all()
    K = fem.assemble_stiffness(act, G, E, NU, Nx, Ny, Nz)
    k, j, i = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    P = np.stack([i.ravel() * G, j.ravel() * G, k.ravel() * G], axis=1).astype(float)
    A = np.array([[0.01, -0.02, 0.005], [0.03, 0.0, -0.01], [0.002, 0.004, 0.02]])
    U = P @ A.T + np.array([0.3, -0.2, 0.1])
    f = (K @ U.ravel()).reshape(-1, 3)
    interior = (i.ravel() > 0) & (i.ravel() < Nx - 1) & (j.ravel() > 0) & (j.ravel() < Ny - 1) & \
        (k.ravel() > 0) & (k.ravel() < Nz - 1)
    assert interior.any()
    assert np.abs(f[interior]).max() < 1e-12
    assert np.abs(f[~interior]).max() > 1e-4  # boundary tractions of the strained block


def test_trilinear_weights_partition_reproduce_linear_and_nodes():
    rng = np.random.default_rng(5)
    for _ in range(50):
        t = rng.random(3)
        w = fem.trilinear_weights(t)
        assert math.isclose(w.sum(), 1.0, rel_tol=1e-15) and (w >= 0).all()
        corners = np.array([fem.local_node(a) for a in range(8)], dtype=float)
        assert np.allclose(w @ corners, t, atol=1e-15)
    for a in range(8):
        w = fem.trilinear_weights(fem.local_node(a))
        assert w[a] == 1.0 and w.sum() == 1.0


def test_block_cell_on_the_last_vertex_plane_and_elementwise_lookup():
    N = fem.grid_nodes((17, 9, 8), 4)
    assert N == (5, 3, 3)
    cell, t = fem.block_cell((16, 8, 7), 4, *N)
    assert cell == (3, 1, 1) and t == (1.0, 1.0, 0.75)
    cell, t = fem.block_cell((5, 0, 3), 4, *N)
    assert cell == (1, 0, 0) and t == (0.25, 0.0, 0.75)


def test_sparse_assembly_equals_dense_loops():
    mask = _mask(9, 9, 9, 0.5)
    g = 3
    Nx, Ny, Nz = fem.grid_nodes((9, 9, 9), g)
    act = fem.active_elements(mask, g)
    assert 0 < act.sum() < act.size
    Ke = fem.element_stiffness(g, E, NU)
    n = 3 * Nx * Ny * Nz
    Kd = np.zeros((n, n))
    for k in range(Nz - 1):
        for j in range(Ny - 1):
            for i in range(Nx - 1):
                if not act[k, j, i]:
                    continue
                for a in range(8):
                    ax, ay, az = fem.local_node(a)
                    na = (i + ax) + Nx * ((j + ay) + Ny * (k + az))
                    for b in range(8):
                        bx, by, bz = fem.local_node(b)
                        nb = (i + bx) + Nx * ((j + by) + Ny * (k + bz))
                        for ca in range(3):
                            for cb in range(3):
                                Kd[3 * na + ca, 3 * nb + cb] += Ke[3 * a + ca, 3 * b + cb]
    K = fem.assemble_stiffness(act, g, E, NU, Nx, Ny, Nz).toarray()
    assert np.allclose(K, Kd, rtol=0, atol=1e-13)


def _blocks(mask, g, n, rng):
    """n distinct block centres (x, y, z) whose element is in the model."""
    nz, ny, nx = mask.shape
    N = fem.grid_nodes((nx, ny, nz), g)
    act = fem.active_elements(mask, g)
    pts = np.argwhere(mask != 0)[:, ::-1]
    ok = [p for p in pts if act[fem.block_cell(p, g, *N)[0][::-1]]]
    pick = rng.choice(len(ok), size=n, replace=False)
    return np.ascontiguousarray(np.array(ok)[pick]).astype(np.int32)


def test_translation_is_recovered_and_nothing_rejected():
    rng = np.random.default_rng(11)
    mask = _mask(24, 20, 16)
    c = _blocks(mask, G, 120, rng)
    t = np.array([2, -1, 3])
    disp = np.tile(t, (len(c), 1)).astype(np.int32)
    ncc = rng.uniform(0.3, 1.0, len(c))
    valid = np.ones(len(c), dtype=np.uint8)
    U, s, rej, _ = fem.update(mask, c, disp, ncc, valid, G, E, NU, n_rej=2, n_int=1, fr=0.1)
    m = fem.Model(mask, c, G, E, NU)
    assert np.allclose(U[m.node_on], t, atol=1e-9)
    assert np.all(U[~m.node_on] == 0)
    assert not rej.any()  # every residual is zero up to rounding: no outlier to reject


def test_affine_field_is_a_fixed_point_of_the_step():
    # D sampled from an affine field A at the blocks: H A = D exactly, so
    # [K + H^T S H] A = H^T S D + K A and one step from U_i = A returns A;
    # dropping F_i = K U_i (or H^T S D) breaks it
    rng = np.random.default_rng(12)
    mask = _mask(24, 20, 16)
    c = _blocks(mask, G, 150, rng)
    m = fem.Model(mask, c, G, E, NU)
    Nx, Ny, Nz = m.N
    k, j, i = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    P = np.stack([i.ravel() * G, j.ravel() * G, k.ravel() * G], axis=1).astype(float)
    A = np.array([[0.05, 0.01, -0.02], [-0.03, 0.04, 0.0], [0.02, 0.0, -0.05]])
    t0 = np.array([1.0, -2.0, 0.5])
    Ua = (P @ A.T + t0) * m.node_on[:, None]
    disp = c.astype(float) @ A.T + t0
    s = fem.confidence(rng.uniform(0.2, 1.0, len(c)), np.ones(len(c)), m.inside)
    U1 = m.step(Ua.ravel(), s, disp).reshape(-1, 3)
    assert np.abs(U1 - Ua).max() < 1e-9
    # and from U = 0 the iteration moves towards it monotonically
    U = np.zeros(Ua.size)
    errs = []
    for _ in range(4):
        U = m.step(U, s, disp)
        errs.append(np.abs(U.reshape(-1, 3) - Ua).max())
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_planted_outliers_are_rejected_first():
    rng = np.random.default_rng(13)
    mask = _mask(32, 28, 20)
    c = _blocks(mask, G, 300, rng)
    disp = np.tile([1, 0, -1], (len(c), 1)).astype(np.int32)
    bad = rng.choice(len(c), size=15, replace=False)
    disp[bad] += rng.choice([-1, 1], size=(15, 3)) * 9
    ncc = rng.uniform(0.5, 1.0, len(c))
    valid = np.ones(len(c), dtype=np.uint8)
    fr = 15 / 300  # floor(0.5 + 300 * 0.05) = 15
    assert fem.n_reject(300, fr) == 15
    U, s, rej, when = fem.update(mask, c, disp, ncc, valid, G, E, NU, n_rej=1, n_int=2, fr=fr)
    assert set(np.nonzero(rej)[0].tolist()) == set(bad.tolist())
    assert (when[bad] == 0).all() and (s[bad] == 0).all()
    # after the rejection the interpolation steps pull the field back to the
    # inliers' translation: their largest residual shrinks step by step
    m = fem.Model(mask, c, G, E, NU)
    good = np.setdiff1d(np.arange(len(c)), bad)
    worst = []
    for n_int in (0, 1, 2, 3):
        U, *_ = fem.update(mask, c, disp, ncc, valid, G, E, NU, n_rej=1, n_int=n_int, fr=fr, model=m)
        worst.append(fem.residuals(m.H, U.ravel(), disp)[good].max())
    assert all(b < a for a, b in zip(worst, worst[1:])), worst


def test_rejection_count_rule_and_ties():
    assert fem.n_reject(10, 0.25) == 3  # floor(0.5 + 2.5)
    assert fem.n_reject(10, 0.24) == 2
    assert fem.n_reject(0, 0.5) == 0
    s = np.array([1.0, 1.0, 0.0, 1.0, 1.0, 1.0])
    r2 = np.array([4.0, 9.0, 100.0, 4.0, 1e-6, 4.0])
    # 5 candidates, F_r = 0.5: floor(3.0) = 3 -> 9, then the first two 4.0 by index
    assert fem.reject(s, r2, 0.5).tolist() == [1, 0, 3]
    # never a residual at or below R2_MIN: F_r = 1 rejects the 4 others only
    assert sorted(fem.reject(s, r2, 1.0).tolist()) == [0, 1, 3, 5]


def test_confidence_reading():
    inside = np.array([True, True, True, False, True])
    s = fem.confidence(np.array([0.5, -0.2, np.nan, 0.9, 0.7]), np.array([1, 1, 0, 1, 0]), inside)
    assert s.tolist() == [0.5, 0.0, 0.0, 0.0, 0.0]


def test_direct_solve_equals_dense_solve():
    rng = np.random.default_rng(14)
    mask = _mask(12, 12, 12, 0.5)
    c = _blocks(mask, 3, 40, rng)
    m = fem.Model(mask, c, 3, E, NU)
    disp = rng.integers(-3, 4, size=(len(c), 3)).astype(float)
    s = fem.confidence(rng.uniform(0.1, 1.0, len(c)), np.ones(len(c)), m.inside)
    U0 = rng.standard_normal(m.K.shape[0]) * m.dof_on
    U = m.step(U0, s, disp)
    on = np.nonzero(m.dof_on)[0]
    A = (m.K + m.H.T @ np.diag(np.repeat(s, 3)) @ m.H)[on][:, on]
    A = np.asarray(A)
    rhs = (m.H.T @ (np.repeat(s, 3) * disp.ravel()) + m.K @ U0)[on]
    assert np.allclose(U[on], np.linalg.solve(A, rhs), rtol=1e-10, atol=1e-10)


def test_step_without_trusted_blocks_keeps_the_field():
    rng = np.random.default_rng(15)
    mask = _mask(16, 16, 12)
    c = _blocks(mask, G, 20, rng)
    m = fem.Model(mask, c, G, E, NU)
    U0 = rng.standard_normal(m.K.shape[0]) * m.dof_on
    assert np.array_equal(m.step(U0, np.zeros(len(c)), np.ones((len(c), 3))), U0)
    # F_r = 1 rejects every block with a residual: the next step keeps U
    disp = rng.integers(-3, 4, size=(len(c), 3))
    U, s, rej, when = fem.update(mask, c, disp, np.ones(len(c)), np.ones(len(c)), G, E, NU, 2, 0, 1.0)
    assert (s == 0).all() and (when == 0).all()
    U1, *_ = fem.update(mask, c, disp, np.ones(len(c)), np.ones(len(c)), G, E, NU, 1, 0, 1.0)
    assert np.array_equal(U, U1)
