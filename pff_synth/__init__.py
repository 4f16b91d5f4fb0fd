"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the phase-field method.  It only produces
the *inputs* a user would hand to the solver: node coordinates, triangle
connectivity, the pre-notch node set, the loaded boundary edges with their
traction vectors, material parameter sets and the batch draws.  Everything is
a deterministic function of its arguments (counter-based SplitMix64 draws),
so the CUDA path and the oracle see bit-identical inputs.

Units are SI throughout (m, Pa, kg/m^3, J/m^2, s).

Workload shapes follow the paper's dynamic crack-branching plate (Sec. 3.3:
100 x 40 mm glass plate, notch to mid-width at mid-height, opposing tractions
on the top and bottom edges) and the glass material of Table 1 (B1/B3 rows).
The paper's meshes are graded Gmsh meshes that are not available; structured
triangulated grids with optional seeded interior jitter stand in for them.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "splitmix64",
    "uniform01",
    "plate",
    "GLASS",
    "config",
    "batch_draws",
]

_MASK = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 output function (Steele, Lea & Flood 2014; Vigna's
    reference formulation): state x is advanced by the golden gamma and the
    result is mixed.  Works on Python ints and on numpy uint64 arrays."""
    if isinstance(x, np.ndarray):
        with np.errstate(over="ignore"):
            z = x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            return z ^ (z >> np.uint64(31))
    z = (int(x) + 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def uniform01(counter):
    """Uniform double in [0, 1) from one SplitMix64 output (top 53 bits)."""
    z = splitmix64(counter)
    if isinstance(z, np.ndarray):
        return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return (z >> 11) * (2.0 ** -53)


# Soda-lime glass of the paper's B1/B3 rows (Table 1): E = 32 GPa, nu = 0.2,
# rho = 2450 kg/m^3, Gc = 3 J/m^2 (0.003 N/mm); residual stiffness eta = 1e-7
# (Sec. 2.1).  The regularisation length is set per mesh (l0 = 2h).
GLASS = dict(E=32.0e9, nu=0.2, rho=2450.0, Gc=3.0, eta=1.0e-7)


def plate(nx, ny, Lx=0.1, Ly=0.04, jitter=0.0, seed=0, traction=1.0e6,
          notch=True):
    """Structured P1 plate on [0, Lx] x [0, Ly] with nx x ny cells.

    Node n = j*(nx+1) + i sits at (i*hx, j*hy).  Quad q = j*nx + i is split
    along its (i,j)-(i+1,j+1) diagonal into triangle 2q = (n00, n10, n11) and
    triangle 2q+1 = (n00, n11, n01); both are counter-clockwise.

    jitter > 0 moves every interior node by (2u-1)*jitter*h per axis, with
    u = uniform01((seed << 32) + 2n + axis); boundary nodes stay put.

    The pre-notch is the node set {j = ny/2, i <= nx/2} (left half of the
    mid-line), on which the damage is held at 1.  The loaded boundary is the
    list of top edges (traction (0, +t)) and bottom edges (traction (0, -t)).

    Returns a dict of numpy arrays: xy (N,2) f64, tri (Ne,3) i32,
    notch (N,) u8, tedges (M,2) i32, tvec (M,2) f64, plus nx, ny, hx, hy, h.
    """
    nx, ny = int(nx), int(ny)
    if nx < 1 or ny < 1:
        raise ValueError("plate needs at least one cell per axis")
    hx, hy = Lx / nx, Ly / ny
    I, J = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="xy")
    I = I.ravel().astype(np.int64)
    J = J.ravel().astype(np.int64)
    x = I * hx
    y = J * hy
    if jitter > 0.0:
        n = J * (nx + 1) + I
        interior = (I > 0) & (I < nx) & (J > 0) & (J < ny)
        base = np.uint64((int(seed) << 32) & _MASK)
        cx = base + (2 * n).astype(np.uint64)
        cy = cx + np.uint64(1)
        ux = uniform01(cx)
        uy = uniform01(cy)
        x = np.where(interior, x + (2.0 * ux - 1.0) * jitter * hx, x)
        y = np.where(interior, y + (2.0 * uy - 1.0) * jitter * hy, y)
    xy = np.stack([x, y], axis=1).astype(np.float64)

    qi, qj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    qi = qi.ravel().astype(np.int64)
    qj = qj.ravel().astype(np.int64)
    n00 = qj * (nx + 1) + qi
    n10 = n00 + 1
    n01 = n00 + (nx + 1)
    n11 = n01 + 1
    tri = np.empty((2 * nx * ny, 3), dtype=np.int32)
    tri[0::2, 0], tri[0::2, 1], tri[0::2, 2] = n00, n10, n11
    tri[1::2, 0], tri[1::2, 1], tri[1::2, 2] = n00, n11, n01

    nmask = np.zeros((nx + 1) * (ny + 1), dtype=np.uint8)
    if notch:
        if ny % 2:
            raise ValueError("the mid-line notch needs an even ny")
        jm = ny // 2
        nmask[jm * (nx + 1) + np.arange(nx // 2 + 1)] = 1

    ib = np.arange(nx, dtype=np.int64)
    top = np.stack([ny * (nx + 1) + ib, ny * (nx + 1) + ib + 1], axis=1)
    bot = np.stack([ib, ib + 1], axis=1)
    tedges = np.concatenate([top, bot]).astype(np.int32)
    tvec = np.zeros((2 * nx, 2), dtype=np.float64)
    tvec[:nx, 1] = traction
    tvec[nx:, 1] = -traction
    return dict(xy=xy, tri=tri, notch=nmask, tedges=tedges, tvec=tvec,
                nx=nx, ny=ny, hx=hx, hy=hy, h=max(hx, hy), Lx=Lx, Ly=Ly)


def material(l0, model="AT2", split="spectral", **over):
    """Glass parameters with the given regularisation length and model."""
    m = dict(GLASS)
    m.update(l0=float(l0), model=model, split=split, plane="strain")
    m.update(over)
    return m


def config(name, split="spectral", model="AT2"):
    """The synthetic workloads, by name.

    plate_100x40   : 100 x 40 cells on 100 x 40 mm (4,141 nodes, 8,000
                     triangles), 200 steps, no jitter.
    plate_1000x1000: 1000 x 1000 cells on 100 x 40 mm (1,002,001 nodes,
                     2,000,000 triangles), interior jitter +-0.1h, seed 0,
                     1,000 steps.
    plate_500x500  : 500 x 500 cells (251,001 nodes), 300 steps, the
                     differentiation workload.
    plate_40x16    : 40 x 16 cells (697 nodes), the small adjoint check.
    Each uses the glass material, l0 = 2h with h = max(hx, hy), t = 1 MPa,
    dt = 0.5 x CFL.
    """
    table = {
        "plate_100x40": dict(nx=100, ny=40, jitter=0.0, steps=200),
        "plate_1000x1000": dict(nx=1000, ny=1000, jitter=0.1, steps=1000),
        "plate_500x500": dict(nx=500, ny=500, jitter=0.1, steps=300),
        "plate_40x16": dict(nx=40, ny=16, jitter=0.0, steps=60),
    }
    c = dict(table[name])
    mesh = plate(c["nx"], c["ny"], jitter=c["jitter"], seed=0)
    mat = material(2.0 * mesh["h"], model=model, split=split)
    return dict(name=name, mesh=mesh, material=mat, steps=c["steps"],
                cfl=0.5, t_ramp=0.05e-6, cg_tol=1e-8)


def sent(n=700, increments=100, u_max=7e-6):
    """Single-edge-notched tension, quasi-static (Sec. 3.5): a 1 x 1 mm
    square of n x n cells, notch on the left half of the mid-line, bottom
    edge clamped, top edge u_x = 0 and u_y = U rising in equal increments to
    u_max (7e-3 mm); E = 210 GPa, nu = 0.3, Gc = 2.7 N/mm (2700 J/m^2),
    l0 = 2h, AT2 with the volumetric-deviatoric split, plane strain.
    bc flags per node: 1 fix u_x, 2 fix u_y, 4 loaded."""
    mesh = plate(n, n, Lx=1e-3, Ly=1e-3, notch=True, traction=0.0)
    N = mesh["xy"].shape[0]
    j = np.arange(N) // (n + 1)
    bc = np.zeros(N, np.uint8)
    bc[j == 0] = 3
    bc[j == n] = 1 | 4
    mat = material(2.0 * mesh["h"], split="amor")
    mat.update(E=210e9, nu=0.3, Gc=2700.0)
    return dict(name=f"sent_{n}", mesh=mesh, material=mat, bc=bc, increments=increments,
                du=u_max / increments, newton_tol=1e-8, cg_tol=1e-8)


def batch_draws(n_plates=64, seed=1):
    """Per-plate draws for the batched workload from one SplitMix64 counter
    stream starting at (seed << 32): nx = 200 + floor(501 u) cells
    (200..700), ny = round(0.4 nx), Gc = 1 + 4u J/m^2, traction
    t = (0.5 + 1.5u) MPa."""
    out = []
    c = (int(seed) << 32) & _MASK
    for _ in range(n_plates):
        u0 = uniform01(c); u1 = uniform01(c + 1); u2 = uniform01(c + 2)
        c += 3
        nx = 200 + int(np.floor(501 * u0))
        ny = int(round(0.4 * nx))
        ny += ny % 2
        out.append(dict(nx=nx, ny=ny, Gc=1.0 + 4.0 * u1,
                        traction=(0.5 + 1.5 * u2) * 1e6))
    return out
