"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's benchmarks (tinyMD, Sec. 6) use FCC lattices with 4 atoms per unit
cell (32^3 cells on one CPU core, 80^3 on one GPU) set up "as in miniMD", with
rc = 2.5 and a 0.3 Verlet buffer.  These generators produce such systems from a
seed.  They hold none of the method's arithmetic (no forces, lists or
integration): only lattice sites, jitter and Maxwell-Boltzmann velocities, so
both the CUDA path and the CPU oracle can be fed the very same arrays.

Recipe (also stated in the design notes):
  * FCC lattice constant a = (4/rho)^(1/3); site order 4*((ix*n+iy)*n+iz)+b with
    basis b in {(0,0,0), (1/2,1/2,0), (1/2,0,1/2), (0,1/2,1/2)} * a.
  * optional uniform jitter in [-j, j] per coordinate (j = 0.05 sigma).
  * velocities ~ N(0, sqrt(T/m)) per component from numpy's PCG64, mean
    momentum removed, then rescaled so that sum m v^2 / (3N - 3) = T exactly.
  * replicas of N atoms that are not 4 n^3: n = ceil((N/4)^(1/3)), box
    L = (N/rho)^(1/3), lattice constant L/n, the first N sites of a seeded
    permutation of the 4 n^3 sites, then jitter.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


@dataclass
class System:
    """Positions/velocities (N x 3, float64) and the periodic box (3,)."""
    pos: np.ndarray
    vel: np.ndarray
    box: np.ndarray
    seed: int = 0

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def fcc_sites(n: int, a: float) -> np.ndarray:
    """All 4 n^3 FCC sites of an n x n x n block of unit cells of side a."""
    ix, iy, iz = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cells = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    sites = cells[:, None, :] + FCC_BASIS[None, :, :]
    return (sites.reshape(-1, 3) * a).astype(np.float64)


def maxwell_boltzmann(n: int, temperature: float, mass: float, rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(0.0, math.sqrt(temperature / mass), size=(n, 3))
    v -= v.mean(axis=0, keepdims=True)
    if n > 1 and temperature > 0:
        t_now = mass * float(np.sum(v * v)) / (3 * n - 3)
        v *= math.sqrt(temperature / t_now)
    return v


def fcc_system(n_cells: int, density: float = 0.8442, temperature: float = 1.44,
               mass: float = 1.0, jitter: float = 0.0, seed: int = 1001) -> System:
    """FCC block of n_cells^3 unit cells (N = 4 n_cells^3)."""
    rng = np.random.default_rng(seed)
    a = (4.0 / density) ** (1.0 / 3.0)
    pos = fcc_sites(n_cells, a)
    if jitter > 0:
        pos = pos + rng.uniform(-jitter, jitter, size=pos.shape)
    L = n_cells * a
    pos = np.mod(pos, L)
    vel = maxwell_boltzmann(pos.shape[0], temperature, mass, rng)
    return System(pos, vel, np.full(3, L), seed)


def replica_system(n_atoms: int, density: float, temperature: float, seed: int,
                   mass: float = 1.0, jitter: float = 0.05) -> System:
    """A replica with an arbitrary atom count: the first N sites of a seeded
    permutation of the smallest FCC block holding N atoms, in a cubic box of
    volume N / density."""
    rng = np.random.default_rng(seed)
    n = math.ceil((n_atoms / 4.0) ** (1.0 / 3.0) - 1e-12)
    while 4 * n ** 3 < n_atoms:
        n += 1
    L = (n_atoms / density) ** (1.0 / 3.0)
    sites = fcc_sites(n, L / n)
    pick = rng.permutation(sites.shape[0])[:n_atoms]
    pos = sites[np.sort(pick)]
    if jitter > 0:
        pos = pos + rng.uniform(-jitter, jitter, size=pos.shape)
    pos = np.mod(pos, L)
    vel = maxwell_boltzmann(n_atoms, temperature, mass, rng)
    return System(pos, vel, np.full(3, L), seed)


def replica_ensemble(n_replicas: int = 256, seed: int = 1004, n_min: int = 500,
                     n_max: int = 20000, rho_range=(0.70, 0.90), t_range=(0.8, 1.6)):
    """Independent replicas: N log-uniform in [n_min, n_max], density and
    temperature uniform in their ranges; replica r uses sub-seed (seed, r)."""
    rng = np.random.default_rng(seed)
    counts = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_replicas))
    counts = np.clip(np.round(counts).astype(np.int64), n_min, n_max)
    rhos = rng.uniform(*rho_range, size=n_replicas)
    temps = rng.uniform(*t_range, size=n_replicas)
    out = []
    for r in range(n_replicas):
        sub = int(np.random.SeedSequence([seed, r]).generate_state(1)[0])
        out.append(replica_system(int(counts[r]), float(rhos[r]), float(temps[r]), sub))
    return out


def uniform_box(n: int, L, seed: int = 7) -> System:
    """n atoms uniform in a box (for neighbour-list tests; no force use)."""
    rng = np.random.default_rng(seed)
    L = np.broadcast_to(np.asarray(L, np.float64), (3,)).copy()
    pos = rng.uniform(0.0, 1.0, size=(n, 3)) * L
    vel = rng.normal(0.0, 1.0, size=(n, 3))
    return System(pos, vel, L, seed)


# Named workloads (seed of workload k is 1000 + k).
WORKLOADS = {
    "fcc8_2048": dict(n_cells=8, jitter=0.0, seed=1001),
    "fcc32_131072": dict(n_cells=32, jitter=0.0, seed=1002),
    "fcc64_1048576": dict(n_cells=64, jitter=0.05, seed=1003),
    "fcc128_8388608": dict(n_cells=128, jitter=0.05, seed=1003),
    "fcc16_16384": dict(n_cells=16, jitter=0.0, seed=1005),
    # the paper's single-GPU workload (Sec. 6: 80^3 unit cells, 2,048,000 atoms)
    "fcc80_2048000": dict(n_cells=80, jitter=0.0, seed=1006),
    # dense granular packing for the contact model of Eq. 3: spheres of
    # diameter 1 on an FCC lattice with nearest-neighbour distance 0.98
    # (12 contacts each), jitter 0.02, cold velocities
    "dem64_1048576": dict(n_cells=64, density=4.0 / (0.98 * 2.0 ** 0.5) ** 3, temperature=0.05,
                          jitter=0.02, seed=1007),
}


def workload(name: str) -> System:
    return fcc_system(**WORKLOADS[name])
