"""Seeded synthetic inputs for the micro-macro KFVS step: grids, parameters, initial states.

This module holds problem set-up only (grids, boundary kinds, seeded initial macro fields in the
conserved form Q = (rho, rho u, rho u (x) u + P), optional seeded g); it contains none of the
scheme's arithmetic.  Both the CUDA path's tests and the oracle's tests draw their inputs from
here.  Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), mapped to doubles by taking the top 53 bits.
"""
from dataclasses import dataclass, field
import math

import numpy as np

PERIODIC, EXTRAP, SPECULAR, DIFFUSE = 0, 1, 2, 3
TAU_RHO, TAU_HARDSPHERE2D, TAU_PRESSURE, TAU_CONST = 0, 1, 2, 3
CFL_MIN, CFL_SUM = 0, 1
PREC_FP64, PREC_G_FP32 = 0, 1

_MASK = (1 << 64) - 1


@dataclass
class Grid:
    nx: int
    ny: int
    x0: float = 0.0
    x1: float = 1.0
    y0: float = 0.0
    y1: float = 1.0
    nv1: int = 8
    nv2: int = 8
    v1min: float = -8.0
    v1max: float = 8.0
    v2min: float = -8.0
    v2max: float = 8.0

    @property
    def ncell(self):
        return self.nx * self.ny

    @property
    def nv(self):
        return self.nv1 * self.nv2

    @property
    def nphase(self):
        return self.nx * self.ny * self.nv1 * self.nv2

    def xc(self):
        dx = (self.x1 - self.x0) / self.nx
        return self.x0 + (np.arange(self.nx) + 0.5) * dx

    def yc(self):
        dy = (self.y1 - self.y0) / self.ny
        return self.y0 + (np.arange(self.ny) + 0.5) * dy

    def v1(self):
        dv = (self.v1max - self.v1min) / self.nv1
        return self.v1min + (np.arange(self.nv1) + 0.5) * dv

    def v2(self):
        dv = (self.v2max - self.v2min) / self.nv2
        return self.v2min + (np.arange(self.nv2) + 0.5) * dv


@dataclass
class Params:
    nu: float = -0.5
    tau_model: int = TAU_RHO
    tau0: float = 1.0
    bc: tuple = (EXTRAP, EXTRAP, EXTRAP, EXTRAP)
    wall_T: tuple = (1.0, 1.0, 1.0, 1.0)
    wall_U: tuple = (0.0, 0.0, 0.0, 0.0)
    wall_keep_es_term: int = 1
    precision: int = PREC_FP64


@dataclass
class Problem:
    grid: Grid
    params: Params
    Q: np.ndarray           # [6][ny][nx]
    G: np.ndarray           # [ny][nx][nv2][nv1]
    eps: float
    dt: float
    nsteps: int
    name: str = ""
    meta: dict = field(default_factory=dict)


class SplitMix64:
    def __init__(self, seed: int):
        self.state = int(seed) & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, lo=0.0, hi=1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on [lo, hi] inclusive."""
        return lo + int(self.uniform() * (hi - lo + 1))

    def array(self, n: int, lo=0.0, hi=1.0) -> np.ndarray:
        """n uniforms in [lo, hi) from a vectorised SplitMix64 stream seeded by this generator."""
        base = np.uint64(self.next_u64())
        with np.errstate(over="ignore"):
            s = base + np.arange(1, n + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
            z = s
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u


def q_from_prims(rho, u1, u2, T, aniso=None, shear=None):
    """Conserved moments Q = (rho, rho u1, rho u2, E11, E12, E22) with P = rho (T I + A), where
    A = [[aniso, shear], [shear, -aniso]] (zero by default: the isotropic initial state)."""
    rho = np.asarray(rho, dtype=np.float64)
    u1 = np.broadcast_to(np.asarray(u1, dtype=np.float64), rho.shape)
    u2 = np.broadcast_to(np.asarray(u2, dtype=np.float64), rho.shape)
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), rho.shape)
    a = np.zeros_like(rho) if aniso is None else np.broadcast_to(np.asarray(aniso, float), rho.shape)
    s = np.zeros_like(rho) if shear is None else np.broadcast_to(np.asarray(shear, float), rho.shape)
    Q = np.empty((6,) + rho.shape)
    Q[0] = rho
    Q[1] = rho * u1
    Q[2] = rho * u2
    Q[3] = rho * u1 * u1 + rho * (T + a)
    Q[4] = rho * u1 * u2 + rho * s
    Q[5] = rho * u2 * u2 + rho * (T - a)
    return np.ascontiguousarray(Q)


def zero_g(grid: Grid) -> np.ndarray:
    return np.zeros((grid.ny, grid.nx, grid.nv2, grid.nv1))


def seeded_g(grid: Grid, seed: int, amp: float = 0.05) -> np.ndarray:
    """Seeded micro part: uniform noise in [-amp, amp] under a unit Gaussian velocity envelope."""
    rng = SplitMix64(seed)
    noise = rng.array(grid.nphase, -amp, amp).reshape(grid.ny, grid.nx, grid.nv2, grid.nv1)
    v1, v2 = grid.v1(), grid.v2()
    env = np.exp(-0.5 * (v2[:, None] ** 2 + v1[None, :] ** 2))
    return np.ascontiguousarray(noise * env[None, None])


def smooth_state(grid: Grid, seed: int, amp: float = 0.2, umax: float = 0.3, aniso: float = 0.1):
    """Seeded smooth periodic macro fields (sum of low Fourier modes) with an anisotropic
    pressure tensor, used for small parity cases."""
    rng = SplitMix64(seed)
    x, y = np.meshgrid(grid.xc(), grid.yc())  # [ny][nx]
    Lx, Ly = grid.x1 - grid.x0, grid.y1 - grid.y0

    def field():
        f = np.zeros_like(x)
        for _ in range(3):
            kx, ky = rng.randint(-2, 2), rng.randint(-2, 2)
            ph = rng.uniform(0, 2 * math.pi)
            f += np.cos(2 * math.pi * (kx * (x - grid.x0) / Lx + ky * (y - grid.y0) / Ly) + ph)
        return f / 3.0

    rho = 1.0 + amp * field()
    T = 1.0 + amp * field()
    u1 = umax * field()
    u2 = umax * field()
    a = aniso * field()
    s = aniso * field()
    return q_from_prims(rho, u1, u2, T, a, s)


# ------------------------------------------------------------------------------------------
# The five workloads of the benchmark family (sizes, boundary kinds, seeds).
# ------------------------------------------------------------------------------------------

def sod_1d2v(nx=200, nv=24, eps=1e-2, cfl=0.5, t_final=0.2) -> Problem:
    """1D-2V Sod shock tube: x in [0,1], ny = 1 with periodic y, v in [-8,8]^2,
    (rho,u,T) = (1,0,1) | (0.125,0,0.8), g = 0, extrapolation in x."""
    grid = Grid(nx=nx, ny=1, nv1=nv, nv2=nv)
    params = Params(nu=-0.5, bc=(EXTRAP, EXTRAP, PERIODIC, PERIODIC))
    x = grid.xc()
    rho = np.where(x < 0.5, 1.0, 0.125)[None, :]
    T = np.where(x < 0.5, 1.0, 0.8)[None, :]
    Q = q_from_prims(rho, 0.0, 0.0, T)
    dt = cfl * ((grid.x1 - grid.x0) / nx) / 8.0
    nsteps = int(math.ceil(t_final / dt * (1 - 1e-12)))
    dt = t_final / nsteps
    return Problem(grid, params, Q, zero_g(grid), eps, dt, nsteps, "sod_1d2v",
                   {"t_final": t_final, "cfl": cfl})


def bump_specular(n=256, nv=32, eps=1e-1, seed=0, cfl=0.5, nsteps=200) -> Problem:
    """2D-2V unit box, specular walls on all sides, rho = 1 + 0.5 exp(-100 |x - x0|^2) with
    x0 ~ U[0.3,0.7]^2 from the seed, u = 0, T = 1, g = 0."""
    grid = Grid(nx=n, ny=n, nv1=nv, nv2=nv)
    params = Params(nu=-0.5, bc=(SPECULAR,) * 4)
    rng = SplitMix64(seed)
    x0, y0 = rng.uniform(0.3, 0.7), rng.uniform(0.3, 0.7)
    x, y = np.meshgrid(grid.xc(), grid.yc())
    rho = 1.0 + 0.5 * np.exp(-100.0 * ((x - x0) ** 2 + (y - y0) ** 2))
    Q = q_from_prims(rho, 0.0, 0.0, 1.0)
    dx = 1.0 / n
    dt = cfl / (8.0 / dx + 8.0 / dx)
    return Problem(grid, params, Q, zero_g(grid), eps, dt, nsteps, "bump_specular",
                   {"seed": seed, "x0": (x0, y0), "cfl": cfl})


def riemann4_diffuse(n=1024, nv=24, eps=1e-2, seed=0, cfl=0.5, nsteps=100, precision=PREC_G_FP32) -> Problem:
    """2D-2V four-quadrant Riemann data split at (0.5, 0.5): per quadrant rho, T ~ U[0.5,1.5],
    u = r (cos th, sin th) with r ~ U[0,0.5], th ~ U[0,2pi); diffuse bottom wall (T_w = 1,
    U_w = 0), extrapolation on the other sides."""
    grid = Grid(nx=n, ny=n, nv1=nv, nv2=nv)
    params = Params(nu=-0.5, bc=(EXTRAP, EXTRAP, DIFFUSE, EXTRAP), precision=precision)
    rng = SplitMix64(seed)
    states = []
    for _ in range(4):
        rho, T = rng.uniform(0.5, 1.5), rng.uniform(0.5, 1.5)
        r, th = rng.uniform(0.0, 0.5), rng.uniform(0.0, 2 * math.pi)
        states.append((rho, r * math.cos(th), r * math.sin(th), T))
    x, y = np.meshgrid(grid.xc(), grid.yc())
    quad = (x >= 0.5).astype(int) + 2 * (y >= 0.5).astype(int)
    f = [np.choose(quad, [s[m] for s in states]) for m in range(4)]
    Q = q_from_prims(f[0], f[1], f[2], f[3])
    dx = 1.0 / n
    dt = cfl / (8.0 / dx + 8.0 / dx)
    return Problem(grid, params, Q, zero_g(grid), eps, dt, nsteps, "riemann4_diffuse",
                   {"seed": seed, "states": states, "cfl": cfl})


def fourier_problem(rng: SplitMix64, nx, ny, nv, eps, cfl=0.5) -> Problem:
    grid = Grid(nx=nx, ny=ny, nv1=nv, nv2=nv)
    params = Params(nu=-0.5, bc=(PERIODIC,) * 4)
    x, y = np.meshgrid(grid.xc(), grid.yc())
    fields = []
    for mean in (1.0, 0.0, 0.0, 1.0):
        f = np.full_like(x, mean)
        for _ in range(4):
            while True:
                kx, ky = rng.randint(-3, 3), rng.randint(-3, 3)
                if (kx, ky) != (0, 0):
                    break
            ph = rng.uniform(0, 2 * math.pi)
            f += (0.2 / 4.0) * np.cos(2 * math.pi * (kx * x + ky * y) + ph)
        fields.append(f)
    Q = q_from_prims(*fields)
    dt = cfl / (8.0 * nx + 8.0 * ny)
    return Problem(grid, params, Q, zero_g(grid), eps, dt, 100, "fourier")


def batch_problems(count=64, seed=0, nmin=64, nmax=256, nvmin=16, nvmax=32):
    """Independent periodic 2D-2V problems of uneven size and eps: nx, ny ~ U{nmin..nmax},
    nv1 = nv2 ~ U{nvmin..nvmax}, eps log-uniform on [1e-3, 1], fields = mean + 0.05 * four
    seeded Fourier modes."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        nx, ny = rng.randint(nmin, nmax), rng.randint(nmin, nmax)
        nv = rng.randint(nvmin, nvmax)
        eps = 10.0 ** rng.uniform(-3.0, 0.0)
        out.append(fourier_problem(rng, nx, ny, nv, eps))
    return out
