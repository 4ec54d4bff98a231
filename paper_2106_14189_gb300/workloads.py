"""Seeded synthetic inputs for the DJ-TLED step: meshes, materials, boundary data.

This module is the one place both the CUDA path and the FP64 oracle take their
inputs from.  It holds no arithmetic of the method itself (no Jacobians,
invariants, forces or time integration): only geometry, connectivity,
material tables and prescribed-displacement lists, generated from a
``numpy.random.default_rng(seed)`` stream so every test and benchmark input is
reproducible.

The workloads stand in for the paper's experiments, whose meshes and image data
are not available:

* ``cube_tet4``: unit cube, Kuhn 6-tet split of an n^3 voxel grid (the paper
  runs T4 meshes of a 0.1 m cube, Sec. 5.1, and a brain of 28764 T4, Sec. 6).
* ``cube_hex8``: unit cube of n^3 8-node bricks (the paper's H8 meshes,
  Sec. 5.1), used with 1-point integration and hourglass control.
* ``ellipsoid_tet4``: brain-sized ellipsoid, two materials, transversely
  isotropic fibres, surface patches displaced as in the brain-shift example
  (Sec. 6: 10-20 mm surface displacements, bottom fixed).
* ``batch_instances``: many boxes of uneven size with random neo-Hookean
  parameters.

Material parameters follow the paper's values: E = 3000 Pa, nu = 0.49
(mu = 1006.712 Pa, kappa = 50000 Pa, Sec. 6) and the conversion used there.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

TET4 = 4
HEX8 = 8

# constitutive model ids (Table 3 rows)
NH, TI, OT, MR = 0, 1, 2, 3

# ramp kinds for prescribed displacements
RAMP_LINEAR = 0    # t / t_total, Sec. 5.1
RAMP_SMOOTH = 1    # C2 quintic 10s^3 - 15s^4 + 6s^5


def lame_from_E_nu(E, nu):
    """Shear and bulk modulus from Young's modulus and Poisson's ratio.

    mu = E / (2 (1 + nu)), kappa = E / (3 (1 - 2 nu)); the paper pairs
    E = 3000 Pa, nu = 0.49 with mu = 1006.712 Pa, kappa = 50000 Pa (Sec. 6).
    """
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    return E / (2.0 * (1.0 + nu)), E / (3.0 * (1.0 - 2.0 * nu))


@dataclass
class Problem:
    """One DJ-TLED problem: mesh, per-element material, prescribed DOFs, run length.

    X      : (N, 3) float64 reference node coordinates [m]
    conn   : (E, n_e) int32 element -> node, 0-based.  T4 nodes follow the
             volume-coordinate order (positive det 0J); H8 nodes are bottom face
             counter-clockwise then top face.
    model  : (E,) uint8 in {NH, TI, OT, MR}
    mu, kappa, rho, eta_a, eta_b, c01 : (E,) float64
             (for MR, C10 = mu / 2 and C01 = c01, Table 3)
    a_dir, b_dir : (E, 3) float64 fibre directions (normalised by the consumer)
    bc_dof : (B,) int64, dof = 3 * node + component
    bc_target : (B,) float64 final prescribed value (0 = fixed)
    """
    name: str
    elem_type: int
    X: np.ndarray
    conn: np.ndarray
    model: np.ndarray
    mu: np.ndarray
    kappa: np.ndarray
    rho: np.ndarray
    eta_a: np.ndarray
    eta_b: np.ndarray
    c01: np.ndarray
    a_dir: np.ndarray
    b_dir: np.ndarray
    bc_dof: np.ndarray
    bc_target: np.ndarray
    n_steps: int = 0
    dt: float = 0.0          # > 0: fixed time step [s]; else dt_scale * dt_crit
    dt_scale: float = 0.9
    alpha: float = 0.0
    hg_coeff: float = 0.1
    ramp_kind: int = RAMP_SMOOTH
    ramp_steps: int = 0
    anp: bool = False        # T4: average nodal pressure in place of the element volumetric term
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.conn.shape[0])


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def _grid_nodes(nx, ny, nz, lx, ly, lz, origin=(0.0, 0.0, 0.0)):
    xs = origin[0] + lx * np.arange(nx + 1) / nx
    ys = origin[1] + ly * np.arange(ny + 1) / ny
    zs = origin[2] + lz * np.arange(nz + 1) / nz
    Z, Y, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([Xg.ravel(), Y.ravel(), Z.ravel()], axis=1)


def _corner_ids(nx, ny, i, j, k):
    sx = nx + 1
    sy = ny + 1
    return i + sx * (j + sy * k)


# The six Kuhn tetrahedra of a voxel: a monotone lattice path from corner
# (0,0,0) to (1,1,1) for each order of the three axes.  All voxels use the same
# diagonal, so the split is conforming across voxel faces.
_KUHN_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
_KUHN_ODD = [False, True, True, False, False, True]


def _kuhn_local():
    """(6, 4, 3) integer corner offsets of the Kuhn tets, positively oriented."""
    out = []
    for perm, odd in zip(_KUHN_PERMS, _KUHN_ODD):
        v = [np.zeros(3, dtype=np.int64)]
        for ax in perm:
            w = v[-1].copy()
            w[ax] += 1
            v.append(w)
        if odd:  # swap the last two vertices to make the orientation positive
            v[2], v[3] = v[3], v[2]
        out.append(np.stack(v))
    return np.stack(out)


def voxel_tets(voxels: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Kuhn split of the listed voxels (V, 3) [i, j, k] -> (6V, 4) corner ids."""
    loc = _kuhn_local()                                   # (6, 4, 3)
    c = voxels[:, None, None, :] + loc[None]              # (V, 6, 4, 3)
    ids = _corner_ids(nx, ny, c[..., 0], c[..., 1], c[..., 2])
    return ids.reshape(-1, 4).astype(np.int64)


def cube_tet4(n: int, L: float = 1.0):
    """Unit-cube style T4 mesh: (n+1)^3 nodes, 6 n^3 Kuhn tets."""
    X = _grid_nodes(n, n, n, L, L, L)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    vox = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    conn = voxel_tets(vox, n, n)
    return X, conn.astype(np.int32)


def box_hex8(nx: int, ny: int, nz: int, lx: float, ly: float, lz: float):
    """Structured H8 box; node order per brick: bottom face CCW, then top face."""
    X = _grid_nodes(nx, ny, nz, lx, ly, lz)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    c = lambda di, dj, dk: _corner_ids(nx, ny, i + di, j + dj, k + dk)
    conn = np.stack([c(0, 0, 0), c(1, 0, 0), c(1, 1, 0), c(0, 1, 0),
                     c(0, 0, 1), c(1, 0, 1), c(1, 1, 1), c(0, 1, 1)], axis=1)
    return X, conn.astype(np.int32)


def box_tet4(nx: int, ny: int, nz: int, lx: float, ly: float, lz: float):
    X = _grid_nodes(nx, ny, nz, lx, ly, lz)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    vox = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    return X, voxel_tets(vox, nx, ny).astype(np.int32)


def cube_hex8(n: int, L: float = 1.0):
    return box_hex8(n, n, n, L, L, L)


def _compact(X, conn):
    used = np.unique(conn)
    remap = -np.ones(X.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.size)
    return X[used], remap[conn].astype(np.int32), used


def jitter_interior(X, conn, frac, h, rng, boundary_mask):
    """Move every non-boundary node by U(-frac h, frac h) per coordinate."""
    d = rng.uniform(-frac * h, frac * h, size=X.shape)
    d[boundary_mask] = 0.0
    return X + d


def boundary_nodes_tet(conn: np.ndarray, n_nodes: int) -> np.ndarray:
    """Nodes on faces that belong to exactly one tet (mesh surface)."""
    faces = np.concatenate([conn[:, [0, 1, 2]], conn[:, [0, 1, 3]],
                            conn[:, [0, 2, 3]], conn[:, [1, 2, 3]]])
    fs = np.sort(faces, axis=1)
    _, idx, cnt = np.unique(fs, axis=0, return_index=True, return_counts=True)
    bf = fs[idx[cnt == 1]]
    mask = np.zeros(n_nodes, dtype=bool)
    mask[bf.ravel()] = True
    return mask


# --------------------------------------------------------------------------
# problems
# --------------------------------------------------------------------------

def _uniform_material(E_count, mu, kappa, rho, model=NH):
    return dict(
        model=np.full(E_count, model, dtype=np.uint8),
        mu=np.full(E_count, mu, dtype=np.float64),
        kappa=np.full(E_count, kappa, dtype=np.float64),
        rho=np.full(E_count, rho, dtype=np.float64),
        eta_a=np.zeros(E_count), eta_b=np.zeros(E_count), c01=np.zeros(E_count),
        a_dir=np.tile([1.0, 0.0, 0.0], (E_count, 1)),
        b_dir=np.tile([0.0, 1.0, 0.0], (E_count, 1)),
    )


def _face_bcs(X, axis, value, tol, comps_targets):
    nodes = np.nonzero(np.abs(X[:, axis] - value) <= tol)[0]
    dofs, tg = [], []
    for comp, target in comps_targets:
        dofs.append(3 * nodes + comp)
        tg.append(np.full(nodes.size, target))
    return np.concatenate(dofs).astype(np.int64), np.concatenate(tg)


def cube_compression_tet4(n: int = 10, n_steps: int = 2000, strain: float = -0.2,
                          E: float = 3000.0, nu: float = 0.49, rho: float = 1000.0,
                          name: Optional[str] = None) -> Problem:
    """Unit cube of 6 n^3 Kuhn tets, base fixed, top face u_z ramped to strain*L.

    n = 10 gives 1331 nodes / 6000 T4.  Only u_z is prescribed on the top face
    (x, y free), as in the paper's ramped extension (Sec. 5.1).
    """
    X, conn = cube_tet4(n)
    mu, kappa = lame_from_E_nu(E, nu)
    mat = _uniform_material(conn.shape[0], float(mu), float(kappa), rho)
    tol = 1e-9
    d0, t0 = _face_bcs(X, 2, 0.0, tol, [(0, 0.0), (1, 0.0), (2, 0.0)])
    d1, t1 = _face_bcs(X, 2, 1.0, tol, [(2, strain)])
    return Problem(name=name or f"tet4_cube_{n}", elem_type=TET4, X=X, conn=conn,
                   bc_dof=np.concatenate([d0, d1]), bc_target=np.concatenate([t0, t1]),
                   n_steps=n_steps, ramp_steps=n_steps, ramp_kind=RAMP_SMOOTH, **mat)


def cube_shear(elem_type: int, n: int, n_steps: int = 5000, shear: float = 0.1,
               E: float = 3000.0, nu: float = 0.49, rho: float = 1000.0,
               hg_coeff: float = 0.1) -> Problem:
    """Unit cube, fixed base, top face sheared u_x = shear*L with u_y = u_z = 0."""
    if elem_type == HEX8:
        X, conn = cube_hex8(n)
    else:
        X, conn = cube_tet4(n)
    mu, kappa = lame_from_E_nu(E, nu)
    mat = _uniform_material(conn.shape[0], float(mu), float(kappa), rho)
    tol = 1e-9
    d0, t0 = _face_bcs(X, 2, 0.0, tol, [(0, 0.0), (1, 0.0), (2, 0.0)])
    d1, t1 = _face_bcs(X, 2, 1.0, tol, [(0, shear), (1, 0.0), (2, 0.0)])
    kind = "hex8" if elem_type == HEX8 else "tet4"
    return Problem(name=f"{kind}_cube_{n}_shear", elem_type=elem_type, X=X, conn=conn,
                   bc_dof=np.concatenate([d0, d1]), bc_target=np.concatenate([t0, t1]),
                   n_steps=n_steps, ramp_steps=n_steps, ramp_kind=RAMP_SMOOTH,
                   hg_coeff=hg_coeff, **mat)


def voxel_hex8(voxels: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Bricks of the listed voxels (V, 3) [i, j, k] -> (V, 8) corner ids
    (bottom face CCW, then top face)."""
    i, j, k = voxels[:, 0], voxels[:, 1], voxels[:, 2]
    c = lambda di, dj, dk: _corner_ids(nx, ny, i + di, j + dj, k + dk)
    return np.stack([c(0, 0, 0), c(1, 0, 0), c(1, 1, 0), c(0, 1, 0),
                     c(0, 0, 1), c(1, 0, 1), c(1, 1, 1), c(0, 1, 1)], axis=1).astype(np.int64)


# materials of the cut-out cube experiment (Sec. 5.1)
CUTOUT_MU, CUTOUT_KAPPA, CUTOUT_RHO, CUTOUT_C01 = 6567.0, 326210.0, 1060.0, 3000.0


def cutout_cube(elem_type: int, n: int, model: int = NH, n_steps: int = 20000,
                extension: float = 0.05, L: float = 0.1, radius: float = 0.025,
                depth: float = 0.03, dt: float = 5e-5) -> Problem:
    """The verification model of Sec. 5.1: a cube of side L with a cylindrical
    recess of the given radius and depth centred on each of the four faces
    normal to x and y, voxelised with n cells per side (Kuhn tets or bricks).
    The back face z = 0 is fixed, the front face z = L is pulled by u_z on a
    linear ramp to `extension` over n_steps steps of dt = 5e-5 s (t = 1 s).
    Materials (Sec. 5.1): NH mu = 6567 Pa, kappa = 326210 Pa; TI eta_a = 2 mu,
    a = x; OT eta_a = eta_b = 2 mu, a = x, b = y; MR C10 = mu / 2,
    C01 = 3000 Pa; rho = 1060 kg/m^3.  The printed recess radius (0.05 m, the
    face's half width) is read as its diameter: radius 0.025 m."""
    h = L / n
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    vox = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    cen = (vox + 0.5) * h
    c = 0.5 * L
    in_x = ((cen[:, 1] - c) ** 2 + (cen[:, 2] - c) ** 2 < radius ** 2) & \
        ((cen[:, 0] < depth) | (cen[:, 0] > L - depth))
    in_y = ((cen[:, 0] - c) ** 2 + (cen[:, 2] - c) ** 2 < radius ** 2) & \
        ((cen[:, 1] < depth) | (cen[:, 1] > L - depth))
    vox = vox[~(in_x | in_y)]
    Xg = _grid_nodes(n, n, n, L, L, L)
    conn = voxel_tets(vox, n, n) if elem_type == TET4 else voxel_hex8(vox, n, n)
    X, conn, _ = _compact(Xg, conn)
    E = conn.shape[0]
    mat = _uniform_material(E, CUTOUT_MU, CUTOUT_KAPPA, CUTOUT_RHO, model)
    if model in (TI, OT):
        mat["eta_a"][:] = 2.0 * CUTOUT_MU
    if model == OT:
        mat["eta_b"][:] = 2.0 * CUTOUT_MU
    if model == MR:
        mat["c01"][:] = CUTOUT_C01
    tol = 1e-9 * L
    d0, t0 = _face_bcs(X, 2, 0.0, tol, [(0, 0.0), (1, 0.0), (2, 0.0)])
    d1, t1 = _face_bcs(X, 2, L, tol, [(2, extension)])
    kind = "hex8" if elem_type == HEX8 else "tet4"
    names = {NH: "nh", TI: "ti", OT: "ot", MR: "mr"}
    return Problem(name=f"{kind}_cutout_{n}_{names[model]}", elem_type=elem_type, X=X, conn=conn,
                   bc_dof=np.concatenate([d0, d1]), bc_target=np.concatenate([t0, t1]),
                   n_steps=n_steps, ramp_steps=n_steps, ramp_kind=RAMP_LINEAR, dt=dt, **mat)


def _smooth_field(rng, pts, n_modes, scale):
    """Sum of seeded random Fourier modes evaluated at pts (P, 3)."""
    k = rng.normal(size=(n_modes, 3)) / scale
    ph = rng.uniform(0, 2 * np.pi, size=n_modes)
    amp = rng.normal(size=(n_modes, 3))
    arg = pts @ k.T + ph                                  # (P, M)
    return np.cos(arg) @ amp                              # (P, 3)


def ellipsoid_tet4(h: float = 1.76e-3, axes=(0.070, 0.055, 0.045), seed: int = 0,
                   n_patches: int = 6, patch_radius: float = 0.015,
                   disp_range=(0.002, 0.010), jitter: float = 0.15,
                   fibres: bool = True) -> Problem:
    """Brain-sized ellipsoid of Kuhn tets with two materials and TI fibres.

    Voxels of size h whose centre lies inside the ellipsoid are split into 6
    tets; interior nodes are jittered by U(-0.15h, 0.15h).  Inner ellipsoid
    (0.6 scale) mu = 3 kPa, outer mu = 1 kPa, nu = 0.49, rho = 1000.  Fibre
    direction: normalised sum of 8 random Fourier modes, fibre stiffness
    eta_a / mu in [2, 5] from a smooth field.  n_patches surface discs of radius
    patch_radius, centred on the upper surface with |x| <= a / 2, get a
    displacement of seeded direction and magnitude in disp_range; nodes with
    z < -0.8 c are fixed.  The brain-shift example of
    Sec. 6 prescribes 10-20 mm surface displacements and a fixed base.
    """
    rng = np.random.default_rng(seed)
    a, b, c = axes
    nx, ny, nz = (int(np.ceil(2 * s / h)) + 2 for s in axes)
    org = np.array([-nx * h / 2, -ny * h / 2, -nz * h / 2])
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cen = np.stack([(i.ravel() + 0.5) * h + org[0], (j.ravel() + 0.5) * h + org[1],
                    (k.ravel() + 0.5) * h + org[2]], axis=1)
    inside = (cen[:, 0] / a) ** 2 + (cen[:, 1] / b) ** 2 + (cen[:, 2] / c) ** 2 < 1.0
    vox = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)[inside]
    conn_full = voxel_tets(vox, nx, ny)
    Xfull = _grid_nodes(nx, ny, nz, nx * h, ny * h, nz * h, origin=tuple(org))
    X, conn, _ = _compact(Xfull, conn_full)
    bmask = boundary_nodes_tet(conn, X.shape[0])
    X = jitter_interior(X, conn, jitter, h, rng, bmask)
    E_count = conn.shape[0]
    cent = X[conn].mean(axis=1)
    inner = (cent[:, 0] / (0.6 * a)) ** 2 + (cent[:, 1] / (0.6 * b)) ** 2 \
        + (cent[:, 2] / (0.6 * c)) ** 2 < 1.0
    mu = np.where(inner, 3000.0, 1000.0)
    nu = 0.49
    kappa = 2.0 * mu * (1.0 + nu) / (3.0 * (1.0 - 2.0 * nu))
    if fibres:
        adir = _smooth_field(rng, cent, 8, 0.04)
        adir /= np.linalg.norm(adir, axis=1, keepdims=True)
        s = _smooth_field(rng, cent, 4, 0.05)[:, 0]
        s = (s - s.min()) / max(s.max() - s.min(), 1e-30)
        eta_a = mu * (2.0 + 3.0 * s)
        model = np.full(E_count, TI, dtype=np.uint8)
    else:
        adir = np.tile([1.0, 0.0, 0.0], (E_count, 1))
        eta_a = np.zeros(E_count)
        model = np.full(E_count, NH, dtype=np.uint8)
    # boundary conditions: fixed base, displaced surface patches
    surf = np.nonzero(bmask)[0]
    fixed = surf[X[surf, 2] < -0.8 * c]
    # patch centres on the upper part of the surface and away from the pointed
    # ends of the long axis (|x| <= a / 2), where the voxelised surface is steepest
    cand = surf[(X[surf, 2] > -0.3 * c) & (np.abs(X[surf, 0]) <= 0.5 * a)]
    centres = X[rng.choice(cand, size=n_patches, replace=False)]
    dirs = rng.normal(size=(n_patches, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    mags = rng.uniform(*disp_range, size=n_patches)
    taken = np.zeros(X.shape[0], dtype=bool)
    taken[fixed] = True
    dofs, tgts = [3 * fixed, 3 * fixed + 1, 3 * fixed + 2], [np.zeros(fixed.size)] * 3
    patch_nodes = []
    for p in range(n_patches):
        d = np.linalg.norm(X[surf] - centres[p], axis=1)
        nodes = surf[(d < patch_radius) & ~taken[surf]]
        taken[nodes] = True
        patch_nodes.append(nodes)
        for comp in range(3):
            dofs.append(3 * nodes + comp)
            tgts.append(np.full(nodes.size, mags[p] * dirs[p, comp]))
    return Problem(name="ellipsoid_tet4", elem_type=TET4, X=X, conn=conn, model=model,
                   mu=mu, kappa=kappa, rho=np.full(E_count, 1000.0), eta_a=eta_a,
                   eta_b=np.zeros(E_count), c01=np.zeros(E_count), a_dir=adir,
                   b_dir=np.tile([0.0, 1.0, 0.0], (E_count, 1)),
                   bc_dof=np.concatenate(dofs).astype(np.int64),
                   bc_target=np.concatenate(tgts), ramp_kind=RAMP_SMOOTH,
                   meta=dict(h=h, axes=axes, seed=seed, surface_nodes=surf, fixed_nodes=fixed,
                             patch_nodes=patch_nodes, patch_centres=centres, patch_radius=patch_radius,
                             patch_dirs=dirs, patch_mags=mags, disp_range=disp_range))


def ellipsoid_load_case(problem: Problem, seed: int) -> np.ndarray:
    """Prescribed targets (ordered as problem.bc_dof) of one seeded load case.

    The fixed base stays fixed; every surface patch gets a displacement of
    seeded direction and magnitude U(disp_range) with the smooth bump profile
    (1 - (r / R)^2)^2 over the patch (r distance to the patch centre), which
    meets the free surface with zero slope at r = R.
    """
    m = problem.meta
    rng = np.random.default_rng(seed)
    X = problem.X
    target_of = {}
    for p, nodes in enumerate(m["patch_nodes"]):
        d = rng.normal(size=3)
        d *= rng.uniform(*m["disp_range"]) / np.linalg.norm(d)
        r = np.linalg.norm(X[nodes] - m["patch_centres"][p], axis=1) / m["patch_radius"]
        w = np.clip(1.0 - r * r, 0.0, 1.0) ** 2
        for comp in range(3):
            for n, v in zip(nodes, w * d[comp]):
                target_of[3 * int(n) + comp] = v
    return np.array([target_of.get(int(dof), 0.0) for dof in problem.bc_dof])


def random_tet_mesh_problem(n_elems_target: int, seed: int, model: int = NH,
                            jitter: float = 0.15) -> Problem:
    """Small jittered box of Kuhn tets with random material; used by tests."""
    rng = np.random.default_rng(seed)
    n = max(1, int(round((n_elems_target / 6.0) ** (1.0 / 3.0))))
    dims = rng.uniform(0.5, 1.5, size=3)
    X, conn = box_tet4(n, n, n, *dims)
    bm = boundary_nodes_tet(conn, X.shape[0])
    X = jitter_interior(X, conn, jitter, dims.min() / n, rng, bm)
    return _random_material_problem(X, conn, TET4, rng, model, f"rand_tet_{seed}")


def random_hex_mesh_problem(n: int, seed: int, model: int = NH) -> Problem:
    rng = np.random.default_rng(seed)
    dims = rng.uniform(0.5, 1.5, size=3)
    X, conn = box_hex8(n, n, n, *dims)
    return _random_material_problem(X, conn, HEX8, rng, model, f"rand_hex_{seed}")


def _random_material_problem(X, conn, et, rng, model, name):
    E_count = conn.shape[0]
    E = rng.uniform(1000.0, 10000.0, size=E_count)
    nu = rng.uniform(0.45, 0.49, size=E_count)
    mu, kappa = lame_from_E_nu(E, nu)
    adir = rng.normal(size=(E_count, 3))
    bdir = rng.normal(size=(E_count, 3))
    eta_a = mu * rng.uniform(1.0, 5.0, size=E_count) if model in (TI, OT) else np.zeros(E_count)
    eta_b = mu * rng.uniform(1.0, 5.0, size=E_count) if model == OT else np.zeros(E_count)
    c01 = mu * rng.uniform(0.1, 0.5, size=E_count) if model == MR else np.zeros(E_count)
    zmin, zmax = X[:, 2].min(), X[:, 2].max()
    tol = 1e-9
    d0, t0 = _face_bcs(X, 2, zmin, tol, [(0, 0.0), (1, 0.0), (2, 0.0)])
    disp = rng.uniform(-0.1, 0.1, size=3) * (zmax - zmin)
    d1, t1 = _face_bcs(X, 2, zmax, tol, [(0, disp[0]), (1, disp[1]), (2, disp[2])])
    return Problem(name=name, elem_type=et, X=X, conn=conn,
                   model=np.full(E_count, model, dtype=np.uint8), mu=mu, kappa=kappa,
                   rho=rng.uniform(900.0, 1100.0, size=E_count), eta_a=eta_a, eta_b=eta_b,
                   c01=c01, a_dir=adir, b_dir=bdir,
                   bc_dof=np.concatenate([d0, d1]), bc_target=np.concatenate([t0, t1]),
                   ramp_kind=RAMP_SMOOTH)


def batch_instances(n_instances: int = 256, seed: int = 0, e_min: int = 5000,
                    e_max: int = 150000, n_steps: int = 2000) -> List[Problem]:
    """Uneven batch: T4/H8 50/50, element count log-uniform in [e_min, e_max].

    Each instance is a box of random aspect with E in U[1, 10] kPa,
    nu in U[0.45, 0.49], rho = 1000, fixed base and a random displacement of
    the top face (or of one side face, scaled by height z / lz).
    """
    rng = np.random.default_rng(seed)
    out = []
    for inst in range(n_instances):
        et = TET4 if rng.uniform() < 0.5 else HEX8
        target = float(np.exp(rng.uniform(np.log(e_min), np.log(e_max))))
        aspect = rng.uniform(0.5, 2.0, size=3)
        per_cell = 6.0 if et == TET4 else 1.0
        cells = target / per_cell
        s = (cells / np.prod(aspect)) ** (1.0 / 3.0)
        nx, ny, nz = (max(1, int(round(s * a))) for a in aspect)
        lx, ly, lz = 0.1 * aspect
        X, conn = (box_tet4 if et == TET4 else box_hex8)(nx, ny, nz, lx, ly, lz)
        E = rng.uniform(1000.0, 10000.0)
        nu = rng.uniform(0.45, 0.49)
        mu, kappa = lame_from_E_nu(E, nu)
        mat = _uniform_material(conn.shape[0], float(mu), float(kappa), 1000.0)
        tol = 1e-12
        d0, t0 = _face_bcs(X, 2, 0.0, tol, [(0, 0.0), (1, 0.0), (2, 0.0)])
        side = int(rng.integers(0, 2))
        disp = rng.uniform(-0.15, 0.15, size=3) * lz
        if side == 0:
            d1, t1 = _face_bcs(X, 2, lz, tol, [(0, disp[0]), (1, disp[1]), (2, disp[2])])
        else:
            # side face x = lx: displacement grows linearly with height so that it
            # is compatible with the fixed base along the shared edge
            d1, t1 = _face_bcs(X, 0, lx, tol, [(0, disp[0]), (1, disp[1]), (2, disp[2])])
            t1 = t1 * X[d1 // 3, 2] / lz
            keep = ~np.isin(d1, d0)
            d1, t1 = d1[keep], t1[keep]
        out.append(Problem(name=f"batch_{inst}", elem_type=et, X=X, conn=conn,
                           bc_dof=np.concatenate([d0, d1]), bc_target=np.concatenate([t0, t1]),
                           n_steps=n_steps, ramp_steps=n_steps, ramp_kind=RAMP_SMOOTH, **mat))
    return out


def single_element(elem_type: int, seed: int = 0, distort: float = 0.2) -> tuple:
    """One randomly distorted, positively oriented element: (X (n_e, 3), conn (1, n_e))."""
    rng = np.random.default_rng(seed)
    if elem_type == TET4:
        base = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    else:
        base = np.array([[-1.0, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                         [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]]) * 0.5
    X = base + rng.uniform(-distort, distort, size=base.shape) * 0.5
    R, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(R) < 0:
        R[:, 0] = -R[:, 0]
    X = X @ R.T * rng.uniform(0.5, 2.0) + rng.normal(size=3)
    conn = np.arange(base.shape[0], dtype=np.int32)[None]
    return X, conn
