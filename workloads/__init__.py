"""Seeded synthetic microstructures for the FFT-Galerkin cell problem.

This module only builds INPUTS: voxel phase maps, per-phase coefficient
tensors, loads and request streams.  It holds none of the method's
arithmetic (no DFT, no projection, no CG), so both the CPU oracle and the
CUDA path can draw their inputs from it without sharing any computation.

Layout conventions (shared by every consumer):
  * a grid is N = (N_1, ..., N_d), every N_a odd (assumption A4 of Sec. 4.1);
  * spatial arrays are C order with the first index slowest;
  * a phase map is uint8 of shape N; a phase table is float64 of shape
    (n_phases, d, d), each entry symmetric positive definite (A1-A2, Sec. 3);
  * a full coefficient field A(x_k) is float64 of shape (d, d, *N).

Geometry is not fixed by the paper (it reports no experiments); the recipes
below follow the workload descriptions (two-phase inclusions, high contrast,
2D and 3D odd grids) and are documented beside each generator.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

SEED_BASE = 13110089


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


@dataclasses.dataclass
class Microstructure:
    """A two- (or more-) phase voxel microstructure on an odd periodic grid."""

    N: Tuple[int, ...]
    phase: np.ndarray          # uint8, shape N
    table: np.ndarray          # float64, (n_phases, d, d)
    name: str = ""
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def d(self) -> int:
        return len(self.N)

    def full_field(self) -> np.ndarray:
        """A(x_k) as a dense (d, d, *N) float64 array (pure gather of the table)."""
        A = self.table[self.phase]                 # (*N, d, d)
        return np.ascontiguousarray(np.moveaxis(A, (-2, -1), (0, 1)))

    def volume_fraction(self, ph: int = 1) -> float:
        return float(np.mean(self.phase == ph))


def isotropic_table(values: Sequence[float], d: int) -> np.ndarray:
    return np.stack([v * np.eye(d) for v in values]).astype(np.float64)


# --------------------------------------------------------------------------
# geometry helpers (periodic distances on integer voxel coordinates)
# --------------------------------------------------------------------------
def _periodic_delta(coord: np.ndarray, centre: float, n: int) -> np.ndarray:
    """Signed minimum-image offset of voxel coordinates from a centre."""
    dlt = coord - centre
    return dlt - n * np.round(dlt / n)


def _stamp_ball(phase: np.ndarray, centre: Sequence[float], radius: float,
                value: int) -> None:
    """Set every voxel whose centre lies within `radius` (periodic) to value."""
    N = phase.shape
    grids = []
    for a, n in enumerate(N):
        lo = int(math.floor(centre[a] - radius)) - 1
        hi = int(math.ceil(centre[a] + radius)) + 2
        idx = np.arange(lo, hi)
        if hi - lo >= n:
            idx = np.arange(n)
        grids.append(idx)
    mesh = np.meshgrid(*grids, indexing="ij")
    dist2 = np.zeros(mesh[0].shape)
    for a, n in enumerate(N):
        dist2 += _periodic_delta(mesh[a].astype(np.float64), centre[a], n) ** 2
    inside = dist2 <= radius * radius
    sel = tuple(np.mod(m[inside], n) for m, n in zip(mesh, N))
    phase[sel] = value


def _periodic_dist(c1, c2, N) -> float:
    s = 0.0
    for a, n in enumerate(N):
        dl = abs(c1[a] - c2[a]) % n
        dl = min(dl, n - dl)
        s += dl * dl
    return math.sqrt(s)


def nonoverlapping_balls(N: Sequence[int], count: int, r_lo: float, r_hi: float,
                         rng: np.random.Generator, max_tries: int = 200000):
    """Seeded centres/radii of `count` balls with periodic distance >= r1+r2."""
    balls: List[Tuple[Tuple[float, ...], float]] = []
    tries = 0
    while len(balls) < count and tries < max_tries:
        tries += 1
        r = float(rng.uniform(r_lo, r_hi))
        c = tuple(float(rng.uniform(0, n)) for n in N)
        if all(_periodic_dist(c, c2, N) >= r + r2 for c2, r2 in balls):
            balls.append((c, r))
    return balls


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def square_inclusion_15() -> Microstructure:
    """15x15 grid, central 7x7 voxels (0-based 4..10) of 10*I in a matrix of 1*I."""
    N = (15, 15)
    phase = np.zeros(N, np.uint8)
    phase[4:11, 4:11] = 1
    return Microstructure(N, phase, isotropic_table([1.0, 10.0], 2),
                          name="square_inclusion_15x15",
                          meta={"contrast": 10.0})


def circles_2d(n: int = 729, count: int = 40, r_lo: float = 10.0,
               r_hi: float = 30.0, contrast: float = 100.0,
               seed: int = SEED_BASE + 1) -> Microstructure:
    """n x n grid with `count` seeded non-overlapping circles (radii U[r_lo,r_hi])."""
    rng = _rng(seed)
    N = (n, n)
    phase = np.zeros(N, np.uint8)
    balls = nonoverlapping_balls(N, count, r_lo, r_hi, rng)
    for c, r in balls:
        _stamp_ball(phase, c, r, 1)
    ms = Microstructure(N, phase, isotropic_table([1.0, contrast], 2),
                        name=f"circles_{n}x{n}",
                        meta={"contrast": contrast, "count": len(balls)})
    ms.meta["vf"] = ms.volume_fraction()
    return ms


def random_spd_pair(d: int, rng: np.random.Generator, lo: float = 1.0,
                    hi: float = 1000.0) -> np.ndarray:
    """Two SPD tensors Q diag(l) Q^T, Q Haar-random, eigenvalues log-uniform in
    [lo, hi], with the smallest eigenvalue overall forced to lo and the largest
    to hi (so that the contrast C_A/c_A of A2 is exactly hi/lo)."""
    out = []
    for ph in range(2):
        g = rng.standard_normal((d, d))
        q, r = np.linalg.qr(g)
        q = q * np.sign(np.diag(r))[None, :]
        lam = np.exp(rng.uniform(math.log(lo), math.log(hi), size=d))
        if ph == 0:
            lam[np.argmin(lam)] = lo
        else:
            lam[np.argmax(lam)] = hi
        out.append(q @ np.diag(lam) @ q.T)
    t = np.stack(out)
    return 0.5 * (t + np.transpose(t, (0, 2, 1)))


def spheres_3d(n: int = 135, count: int = 60, r_lo: float = 6.0,
               r_hi: float = 14.0, seed: int = SEED_BASE + 2,
               anisotropic: bool = True, contrast: float = 1000.0) -> Microstructure:
    """n^3 grid with seeded non-overlapping spheres; two random SPD phases."""
    rng = _rng(seed)
    N = (n, n, n)
    phase = np.zeros(N, np.uint8)
    balls = nonoverlapping_balls(N, count, r_lo, r_hi, rng)
    for c, r in balls:
        _stamp_ball(phase, c, r, 1)
    if anisotropic:
        table = random_spd_pair(3, rng, 1.0, contrast)
    else:
        table = isotropic_table([1.0, contrast], 3)
    ms = Microstructure(N, phase, table, name=f"spheres_{n}^3",
                        meta={"contrast": contrast, "count": len(balls)})
    ms.meta["vf"] = ms.volume_fraction()
    return ms


def _stamp_ellipse(phase: np.ndarray, c0: float, c1: float, a: float, b: float,
                   th: float, value: int) -> None:
    """Set the voxels inside a periodic ellipse (centre, semi-axes a >= b, angle)."""
    n0, n1 = phase.shape
    R = int(math.ceil(a)) + 1
    i = np.arange(int(math.floor(c0)) - R, int(math.floor(c0)) + R + 2)
    j = np.arange(int(math.floor(c1)) - R, int(math.floor(c1)) + R + 2)
    ii, jj = np.meshgrid(i, j, indexing="ij")
    d0 = _periodic_delta(ii.astype(np.float64), c0, n0)
    d1 = _periodic_delta(jj.astype(np.float64), c1, n1)
    u = math.cos(th) * d0 + math.sin(th) * d1
    v = -math.sin(th) * d0 + math.cos(th) * d1
    inside = (u / a) ** 2 + (v / b) ** 2 <= 1.0
    phase[np.mod(ii[inside], n0), np.mod(jj[inside], n1)] = value


def ellipses_2d(n: int, vf_target: float, contrast: float,
                rng: np.random.Generator, max_inclusions: int = 10000) -> Microstructure:
    """Overlapping random ellipses added until the phase-1 fraction >= vf_target."""
    N = (n, n)
    phase = np.zeros(N, np.uint8)
    k = 0
    while phase.mean() < vf_target and k < max_inclusions:
        k += 1
        a = rng.uniform(0.03, 0.12) * n
        b = a * rng.uniform(0.3, 1.0)
        th = rng.uniform(0, math.pi)
        c0, c1 = rng.uniform(0, n), rng.uniform(0, n)
        _stamp_ellipse(phase, c0, c1, a, b, th, 1)
    ms = Microstructure(N, phase, isotropic_table([1.0, contrast], 2),
                        name=f"ellipses_{n}x{n}",
                        meta={"contrast": contrast, "vf_target": vf_target})
    ms.meta["vf"] = ms.volume_fraction()
    return ms


BATCH_SIZES = (45, 75, 135, 243, 375)


def batch_2d(count: int = 256, seed: int = SEED_BASE + 3,
             sizes: Sequence[int] = BATCH_SIZES) -> List[Microstructure]:
    """Independent 2D problems: size uniform over `sizes`, vf ~ U[0.1,0.5],
    contrast log-uniform over [10, 1e4]."""
    rng = _rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice(sizes))
        vf = float(rng.uniform(0.1, 0.5))
        c = float(math.exp(rng.uniform(math.log(10.0), math.log(1.0e4))))
        out.append(ellipses_2d(n, vf, c, rng))
    return out


SERVING_GRIDS = ((81, 81), (243, 243), (729, 729), (27, 27, 27), (45, 45, 45),
                 (81, 81, 81), (135, 135, 135))


def balls_to_vf(N: Sequence[int], vf: float, rng: np.random.Generator,
                contrast: float) -> Microstructure:
    """Overlapping circles/spheres (radius ~ U[0.04,0.1]*min N) until vf."""
    phase = np.zeros(tuple(N), np.uint8)
    nmin = min(N)
    k = 0
    while phase.mean() < vf and k < 100000:
        k += 1
        r = float(rng.uniform(0.04, 0.1)) * nmin
        c = tuple(float(rng.uniform(0, n)) for n in N)
        _stamp_ball(phase, c, max(r, 1.0), 1)
    d = len(N)
    ms = Microstructure(tuple(N), phase, isotropic_table([1.0, contrast], d),
                        name="balls_" + "x".join(map(str, N)),
                        meta={"contrast": contrast})
    ms.meta["vf"] = ms.volume_fraction()
    return ms


@dataclasses.dataclass
class Request:
    t_arrival: float
    ms: Microstructure


def serving_stream(duration_s: float = 60.0, rate: float = 200.0,
                   seed: int = SEED_BASE + 4,
                   grids: Sequence[Tuple[int, ...]] = SERVING_GRIDS,
                   max_requests: Optional[int] = None,
                   cache: bool = True) -> List[Request]:
    """Poisson arrivals (seeded exponential gaps) of random two-phase problems.

    With cache=True, microstructures are drawn from a small seeded pool per
    grid size (8 each) so that generating a long stream stays cheap; the
    arrival order, sizes and contrasts are still random per request."""
    rng = _rng(seed)
    pool = {}
    out: List[Request] = []
    t = 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration_s:
            break
        if max_requests is not None and len(out) >= max_requests:
            break
        g = tuple(grids[int(rng.integers(len(grids)))])
        c = float(math.exp(rng.uniform(math.log(10.0), math.log(1.0e3))))
        slot = int(rng.integers(8))
        key = (g, slot)
        if not cache or key not in pool:
            base = balls_to_vf(g, 0.2, _rng(seed * 31 + hash(key) % 100003), 1.0)
            pool[key] = base
        base = pool[key]
        ms = Microstructure(base.N, base.phase,
                            isotropic_table([1.0, c], len(g)),
                            name=base.name, meta={"contrast": c, "vf": base.meta["vf"]})
        out.append(Request(t, ms))
    return out


def laminate(N: Sequence[int], values_along_axis0: Sequence[float]) -> Microstructure:
    """A(x) = a(x_1) I, varying only along the first axis (one phase per layer)."""
    vals = list(values_along_axis0)
    assert len(vals) == N[0]
    uniq = sorted(set(vals))
    if len(uniq) > 255:
        raise ValueError("too many distinct layer values for a uint8 phase map")
    phase = np.zeros(tuple(N), np.uint8)
    for i, v in enumerate(vals):
        phase[i, ...] = uniq.index(v)
    return Microstructure(tuple(N), phase, isotropic_table(uniq, len(N)),
                          name="laminate")


def random_spd_field(N: Sequence[int], rng: np.random.Generator,
                     lo: float = 1.0, hi: float = 10.0) -> np.ndarray:
    """Independent random SPD tensor per voxel, eigenvalues in [lo, hi]: (d,d,*N)."""
    d = len(N)
    M = int(np.prod(N))
    g = rng.standard_normal((M, d, d))
    q, _ = np.linalg.qr(g)
    lam = rng.uniform(lo, hi, size=(M, d))
    A = np.einsum("mij,mj,mkj->mik", q, lam, q)
    A = 0.5 * (A + np.transpose(A, (0, 2, 1)))
    return np.ascontiguousarray(np.moveaxis(A.reshape(tuple(N) + (d, d)), (-2, -1), (0, 1)))


def unit_loads(d: int) -> np.ndarray:
    """Macroscopic loads E = e_1 ... e_d (Eq. grad_field_split), shape (d, d)."""
    return np.eye(d)
