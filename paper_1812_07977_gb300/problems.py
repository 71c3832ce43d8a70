"""Seeded synthetic inputs: initial conditions for the RiemannProblem family.

This module serves both the CUDA path and the CPU oracle.  It holds problem
set-up only (cell centres, the states either side of an interface, seeded
random numbers, the ideal-gas energy of the initial data) and none of the
finite-volume step's arithmetic.  Every generator returns the INTERIOR
conserved state as a C-contiguous float64 array of shape (5, nz, ny, nx):
rho, rho*vx, rho*vy, rho*vz, E, with x fastest.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4

# Sod (1978) shock tube states, the RiemannProblem of Sec. 3.
SOD_LEFT = (1.0, 0.0, 1.0)     # rho, normal velocity, p
SOD_RIGHT = (0.125, 0.0, 0.1)

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator; ``uniform(n)`` gives doubles in [0, 1) from the
    top 53 bits of each output."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & _M64)

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            inc = np.uint64(0x9E3779B97F4A7C15)
            z = self.state + inc * np.arange(1, n + 1, dtype=np.uint64)
            self.state = self.state + inc * np.uint64(n)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def cell_centres(n: int, length: float = 1.0) -> np.ndarray:
    """x_i = (i + 1/2) * dx, dx = length / n, for i = 0 .. n-1."""
    dx = length / n
    return (np.arange(n, dtype=np.float64) + 0.5) * dx


def conserved_from_primitive(rho, vx, vy, vz, p, gamma=GAMMA) -> np.ndarray:
    """Initial data: U = (rho, rho v, p/(gamma-1) + rho |v|^2 / 2), stacked."""
    rho, vx, vy, vz, p = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64)
                                               for a in (rho, vx, vy, vz, p)))
    U = np.empty((5,) + rho.shape)
    U[0] = rho
    U[1] = rho * vx
    U[2] = rho * vy
    U[3] = rho * vz
    U[4] = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return np.ascontiguousarray(U)


def _grid(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0):
    z = cell_centres(nz, lz)[:, None, None]
    y = cell_centres(ny, ly)[None, :, None]
    x = cell_centres(nx, lx)[None, None, :]
    return x, y, z


def riemann_planar(nx, ny, nz, axis=0, left=SOD_LEFT, right=SOD_RIGHT, x0=0.5,
                   gamma=GAMMA) -> np.ndarray:
    """Planar Riemann problem normal to `axis` in the unit cube: the left state
    where the cell centre's coordinate is < x0 (Sod by default, Sec. 3)."""
    x, y, z = _grid(nx, ny, nz)
    s = (x, y, z)[axis] + 0.0 * (x + y + z)
    is_left = s < x0
    rho = np.where(is_left, left[0], right[0])
    vn = np.where(is_left, left[1], right[1])
    p = np.where(is_left, left[2], right[2])
    v = [np.zeros_like(rho) for _ in range(3)]
    v[axis] = vn
    return conserved_from_primitive(rho, v[0], v[1], v[2], p, gamma)


def riemann_oblique(nx, ny, nz, left=SOD_LEFT, right=SOD_RIGHT, gamma=GAMMA,
                    planes=None) -> np.ndarray:
    """Sod states split by the plane through (1/2,1/2,1/2) with normal
    (1,1,1)/sqrt(3): left where (x-1/2)+(y-1/2)+(z-1/2) < 0.  The velocity
    (along the normal) is zero in both Sod states.  planes=(k0, k1): only the
    z planes k0 .. k1-1 of that state (a slab, without building the rest)."""
    x, y, z = _grid(nx, ny, nz)
    if planes is not None:
        z = z[planes[0]:planes[1]]
    s = (x - 0.5) + (y - 0.5) + (z - 0.5)
    is_left = s < 0.0
    rho = np.where(is_left, left[0], right[0])
    vn = np.where(is_left, left[1], right[1])
    p = np.where(is_left, left[2], right[2])
    r3 = 1.0 / math.sqrt(3.0)
    return conserved_from_primitive(rho, vn * r3, vn * r3, vn * r3, p, gamma)


def uniform(nx, ny, nz, rho, v, p, gamma=GAMMA) -> np.ndarray:
    shape = (nz, ny, nx)
    return conserved_from_primitive(np.full(shape, rho), np.full(shape, v[0]),
                                    np.full(shape, v[1]), np.full(shape, v[2]),
                                    np.full(shape, p), gamma)


def random_states(seed: int, n: int, log_lo=-1.0, log_hi=1.0, vmax=1.0):
    """n random primitive states: rho, p log-uniform in [10^log_lo, 10^log_hi],
    v uniform in the ball |v| <= vmax.  Returns (n, 5) rows (rho, vx, vy, vz, p)."""
    g = SplitMix64(seed)
    rho = 10.0 ** (log_lo + (log_hi - log_lo) * g.uniform(n))
    p = 10.0 ** (log_lo + (log_hi - log_lo) * g.uniform(n))
    # uniform in the ball: direction from a normalised cube sample by rejection
    v = np.empty((n, 3))
    filled = 0
    while filled < n:
        c = 2.0 * g.uniform(3 * n).reshape(n, 3) - 1.0
        ok = c[(c * c).sum(1) <= 1.0]
        take = min(len(ok), n - filled)
        v[filled:filled + take] = ok[:take] * vmax
        filled += take
    return np.column_stack([rho, v, p])


def random_smooth_periodic(nx, ny, nz, seed: int, amp=0.2, gamma=GAMMA) -> np.ndarray:
    """A smooth periodic state from a few random Fourier modes (seeded):
    rho, p in [1-amp, 1+amp] scaled, |v| <= 0.5."""
    g = SplitMix64(seed)
    x, y, z = _grid(nx, ny, nz)
    fields = []
    for f in range(5):
        acc = np.zeros((nz, ny, nx))
        for _ in range(3):
            k = np.floor(g.uniform(3) * 3.0) + 1.0
            ph = 2.0 * math.pi * g.uniform(1)[0]
            acc = acc + np.sin(2.0 * math.pi * (k[0] * x + k[1] * y + k[2] * z) + ph)
        fields.append(acc / 3.0)
    rho = 1.0 + amp * fields[0]
    p = 1.0 + amp * fields[4]
    return conserved_from_primitive(rho, 0.5 * fields[1], 0.5 * fields[2],
                                    0.5 * fields[3], p, gamma)


def entropy_wave_1d(n: int, amp=0.2, velocity=1.0, p=1.0, gamma=GAMMA) -> np.ndarray:
    """Exact cell averages of rho = 1 + amp sin(2 pi x), v = (velocity,0,0),
    p const, on n x 1 x 1 cells of the unit interval (periodic in x)."""
    dx = 1.0 / n
    x = cell_centres(n)
    sinc = math.sin(math.pi * dx) / (math.pi * dx)
    rho = 1.0 + amp * sinc * np.sin(2.0 * math.pi * x)
    rho = rho.reshape(1, 1, n)
    U = np.empty((5, 1, 1, n))
    U[0] = rho
    U[1] = rho * velocity
    U[2] = 0.0
    U[3] = 0.0
    U[4] = p / (gamma - 1.0) + 0.5 * velocity * velocity * rho
    return U


def entropy_wave_3d(n: int, amp=0.2, p=1.0, gamma=GAMMA) -> np.ndarray:
    """Exact cell averages of rho = 1 + amp sin(2 pi (x+y+z)), v = (1,1,1),
    p const on an n^3 periodic unit cube.  At t = 1/3 the exact solution
    equals the initial data."""
    dx = 1.0 / n
    x, y, z = _grid(n, n, n)
    sinc = math.sin(math.pi * dx) / (math.pi * dx)
    rho = 1.0 + amp * sinc ** 3 * np.sin(2.0 * math.pi * (x + y + z))
    U = np.empty((5, n, n, n))
    U[0] = rho
    U[1] = rho
    U[2] = rho
    U[3] = rho
    U[4] = p / (gamma - 1.0) + 1.5 * rho
    return U


def riemann_random_plane(nx, ny, nz, left, right, normal, gamma=GAMMA) -> np.ndarray:
    """Riemann problem split by the plane through the cube centre with unit
    `normal`: primitive states left = (rho, v(3), p) where
    (x - 1/2, y - 1/2, z - 1/2) . normal < 0, right elsewhere.  The unit cube
    is covered by nx x ny x nz cells (dx differs per axis when they differ)."""
    x, y, z = _grid(nx, ny, nz)
    s = (x - 0.5) * normal[0] + (y - 0.5) * normal[1] + (z - 0.5) * normal[2]
    is_left = s < 0.0
    f = [np.where(is_left, left[q], right[q]) for q in range(5)]
    return conserved_from_primitive(f[0], f[1], f[2], f[3], f[4], gamma)


def batched_riemann(seed: int = 12345, count: int = 96,
                    lengths=tuple(range(16, 129, 8))):
    """The batched workload: `count` meshes, each axis length drawn uniformly
    from {16, 24, ..., 128}; each mesh a Riemann problem with rho and p
    log-uniform in [0.1, 10] on either side, velocities uniform in the unit
    ball, and a plane normal uniform on the sphere.  Returns a list of dicts
    with the shape (nx, ny, nz), the states, the normal and U0."""
    g = SplitMix64(seed)
    out = []
    L = np.array(lengths)
    for _ in range(count):
        n = [int(L[min(int(u * len(L)), len(L) - 1)]) for u in g.uniform(3)]
        rho = 10.0 ** (-1.0 + 2.0 * g.uniform(2))
        p = 10.0 ** (-1.0 + 2.0 * g.uniform(2))
        vel = []
        while len(vel) < 2:
            c = 2.0 * g.uniform(3) - 1.0
            if float(c @ c) <= 1.0:
                vel.append(c)
        while True:
            c = 2.0 * g.uniform(3) - 1.0
            r2 = float(c @ c)
            if 1e-6 < r2 <= 1.0:
                normal = c / math.sqrt(r2)
                break
        left = (rho[0], *vel[0], p[0])
        right = (rho[1], *vel[1], p[1])
        out.append({"shape": tuple(n), "left": left, "right": right, "normal": normal,
                    "U0": riemann_random_plane(*n, left, right, normal)})
    return out


def shear_layer(n: int, amp: float, gamma: float = GAMMA, p0: float = 2.5,
                modes=None, seed: int = 0) -> np.ndarray:
    """Periodic shear layer on an n^3 unit cube: rho = 2, vx = +0.5 for
    |y - 1/2| < 1/4, rho = 1, vx = -0.5 elsewhere, p = p0, and the
    perturbation vy = amp sin(4 pi x) (the same in every z plane).  With
    `modes` > 0 the perturbation is instead a seeded sum of that many modes
    with integer wave vectors in {1..4}^3 and random phases, of total
    amplitude amp, on vy and vz."""
    x, y, z = _grid(n, n, n)
    inside = np.abs(y - 0.5) < 0.25
    rho = np.where(inside, 2.0, 1.0) + 0.0 * (x + z)
    vx = np.where(inside, 0.5, -0.5) + 0.0 * (x + z)
    if not modes:
        vy = amp * np.sin(4.0 * math.pi * x) + 0.0 * (y + z)
        vz = np.zeros_like(rho)
    else:
        g = SplitMix64(seed)
        vy = np.zeros_like(rho)
        vz = np.zeros_like(rho)
        for _ in range(modes):
            k = np.floor(g.uniform(3) * 4.0) + 1.0
            ph = 2.0 * math.pi * g.uniform(2)
            arg = 2.0 * math.pi * (k[0] * x + k[1] * y + k[2] * z)
            vy = vy + np.sin(arg + ph[0])
            vz = vz + np.sin(arg + ph[1])
        vy *= amp / modes
        vz *= amp / modes
    return conserved_from_primitive(rho, vx, vy, vz, np.full_like(rho, p0), gamma)



def shear_layer_device(n: int, amp: float, gamma: float = GAMMA, p0: float = 2.5,
                       modes: int = 8, seed: int = 0, device="cuda"):
    """shear_layer(n, amp, gamma, p0, modes, seed) built on a torch device
    (the same seeded draws and formulas; for meshes too large to build on
    the host).  Returns a contiguous float64 tensor (5, n, n, n)."""
    import torch
    c = (torch.arange(n, dtype=torch.float64, device=device) + 0.5) / n
    z, y, x = c[:, None, None], c[None, :, None], c[None, None, :]
    inside = (y - 0.5).abs() < 0.25
    shape = (n, n, n)
    rho = torch.where(inside, 2.0, 1.0).expand(shape)
    vx = torch.where(inside, 0.5, -0.5).expand(shape)
    g = SplitMix64(seed)
    vy = torch.zeros(shape, dtype=torch.float64, device=device)
    vz = torch.zeros(shape, dtype=torch.float64, device=device)
    for _ in range(modes):
        k = np.floor(g.uniform(3) * 4.0) + 1.0
        ph = 2.0 * math.pi * g.uniform(2)
        arg = 2.0 * math.pi * (float(k[0]) * x + float(k[1]) * y + float(k[2]) * z)
        vy += torch.sin(arg + float(ph[0]))
        vz += torch.sin(arg + float(ph[1]))
    vy *= amp / modes
    vz *= amp / modes
    U = torch.empty((5,) + shape, dtype=torch.float64, device=device)
    U[0] = rho
    U[1] = rho * vx
    U[2] = rho * vy
    U[3] = rho * vz
    U[4] = p0 / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return U
