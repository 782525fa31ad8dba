"""Seeded synthetic inputs for the pressure solve: grids, density profiles, sources.

This module holds input generation only. It contains none of the solver's
arithmetic (no coefficients, no projection, no transforms), so that both the
CUDA path and the FP64 CPU oracle can be fed the same arrays without sharing
any code of the method itself.

The paper drives its solvers with MONC's dry boundary-layer test case (Section 3),
which is not available here. The workloads below stand in for it: horizontally
periodic fields on a uniform x/y mesh, stretched vertical levels and an
anelastic reference density that decays with height, at MONC-like local sizes.

Fields are numpy float64 arrays of shape (nz, ny, nx), x fastest.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


@dataclass
class Domain:
    """One pressure-solve problem: grid, vertical levels, density and source."""
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: np.ndarray            # (nz,) cell thicknesses [m]
    rho0: np.ndarray          # (nz,) reference density at cell centres [kg/m^3]
    S: np.ndarray | None = None   # (nz, ny, nx) source
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def npoints(self) -> int:
        return self.nx * self.ny * self.nz


def cell_centres(dz: np.ndarray) -> np.ndarray:
    """Heights of the cell centres for cell thicknesses dz (bottom face at z=0)."""
    dz = np.asarray(dz, dtype=np.float64)
    return np.cumsum(dz) - 0.5 * dz


def stretched_levels(nz: int, dz0: float = 10.0, q: float = 1.03) -> np.ndarray:
    """Geometric level thicknesses dz_k = dz0 * q**k."""
    return dz0 * q ** np.arange(nz, dtype=np.float64)


def exponential_density(dz: np.ndarray, rho_s: float = 1.2, H: float = 8000.0) -> np.ndarray:
    """rho0 evaluated at the cell centres: rho_s * exp(-z/H)."""
    return rho_s * np.exp(-cell_centres(dz) / H)


def normal_source(shape, seed: int, std: float = 1.0) -> np.ndarray:
    """Seeded N(0, std^2) field with its plain mean removed."""
    rng = np.random.default_rng(seed)
    S = rng.standard_normal(shape) * std
    return S - S.mean()


def _periodic_gauss(n: int, centre: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """(nblobs, n) Gaussian profiles on a periodic index axis (minimum-image distance)."""
    idx = np.arange(n, dtype=np.float64)[None, :]
    d = np.abs(idx - centre[:, None])
    d = np.minimum(d, n - d)
    return np.exp(-0.5 * (d / sigma[:, None]) ** 2)


def _open_gauss(n: int, centre: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    idx = np.arange(n, dtype=np.float64)[None, :]
    d = idx - centre[:, None]
    return np.exp(-0.5 * (d / sigma[:, None]) ** 2)


def blob_source(nx: int, ny: int, nz: int, seed: int, nblobs: int = 200,
                sigma_range=(2.0, 10.0), noise_std: float = 0.1) -> np.ndarray:
    """Sum of seeded isotropic Gaussian blobs plus white noise, plain mean removed.

    Amplitudes N(0,1); centres uniform over cell indices; sigma ~ U[2,10] cells,
    isotropic in index space; periodic wrap in x and y, truncated in z; plus
    N(0, noise_std^2) per cell.  An isotropic Gaussian factorises into x, y and
    z profiles, so the field is accumulated as a contraction over blobs.
    """
    rng = np.random.default_rng(seed)
    amp = rng.standard_normal(nblobs)
    cx = rng.uniform(0, nx, nblobs)
    cy = rng.uniform(0, ny, nblobs)
    cz = rng.uniform(0, nz, nblobs)
    sig = rng.uniform(sigma_range[0], sigma_range[1], nblobs)
    gx = _periodic_gauss(nx, cx, sig)            # (b, nx)
    gy = _periodic_gauss(ny, cy, sig)            # (b, ny)
    gz = _open_gauss(nz, cz, sig) * amp[:, None]  # (b, nz)
    S = np.empty((nz, ny, nx))
    for k in range(nz):
        S[k] = (gy * gz[:, k][:, None]).T @ gx
    S += rng.standard_normal(S.shape) * noise_std
    return S - S.mean()


# ---------------------------------------------------------------------------
# The five workloads.  Names describe the problem; sizes are in the names.
# ---------------------------------------------------------------------------

def uniform_cube(n: int = 32, seed: int = 1) -> Domain:
    """n^3 cube, dx=dy=dz=1, constant density, S ~ N(0,1) mean removed (FP64 solve)."""
    dz = np.ones(n)
    rho = np.ones(n)
    return Domain(n, n, n, 1.0, 1.0, dz, rho, normal_source((n, n, n), seed),
                  name=f"uniform_{n}x{n}x{n}_fp64")


def anelastic_blobs(nx: int = 256, ny: int = 256, nz: int = 64, seed: int = 2,
                    with_source: bool = True) -> Domain:
    """dx=dy=50 m, dz_k=10*1.03^k m, rho0=1.2*exp(-z/8000); 200 blobs + N(0,0.1) noise."""
    dz = stretched_levels(nz)
    rho = exponential_density(dz)
    S = blob_source(nx, ny, nz, seed) if with_source else None
    return Domain(nx, ny, nz, 50.0, 50.0, dz, rho, S,
                  name=f"anelastic_blobs_{nx}x{ny}x{nz}")


def anelastic_noise(nx: int = 1024, ny: int = 1024, nz: int = 128, seed: int = 3,
                    with_source: bool = True) -> Domain:
    """Same stretched/anelastic setup, S ~ N(0,1) mean removed (mixed-precision solve)."""
    dz = stretched_levels(nz)
    rho = exponential_density(dz)
    S = normal_source((nz, ny, nx), seed) if with_source else None
    return Domain(nx, ny, nz, 50.0, 50.0, dz, rho, S,
                  name=f"anelastic_noise_{nx}x{ny}x{nz}")


def gradient_problem(nx: int = 512, ny: int = 512, nz: int = 64, seed_S: int = 4,
                     seed_w: int = 5, seed_fd: int = 6, n_fd: int = 32) -> Domain:
    """Blob source (seed 4), loss weights w ~ N(0,1) (seed 5), 32 FD probe indices (seed 6)."""
    d = anelastic_blobs(nx, ny, nz, seed=seed_S)
    rng_w = np.random.default_rng(seed_w)
    w = rng_w.standard_normal((nz, ny, nx))
    rng_fd = np.random.default_rng(seed_fd)
    flat = rng_fd.choice(nx * ny * nz, size=n_fd, replace=False)
    d.extra["w"] = w
    d.extra["fd_index"] = np.sort(flat)
    d.name = f"gradient_{nx}x{ny}x{nz}"
    return d


BATCH_NXY = (64, 128, 256, 384, 512)
BATCH_NZ = (32, 48, 64, 96)
BATCH_DXY = (25.0, 50.0, 100.0)


def uneven_batch(ndomains: int = 64, seed: int = 7, with_source: bool = True,
                 nxy_choices=BATCH_NXY, nz_choices=BATCH_NZ) -> list[Domain]:
    """Independent domains of uneven sizes with seeded stretched levels and density profiles.

    nx=ny from {64,128,256,384,512}, nz from {32,48,64,96}, dx=dy from {25,50,100} m,
    dz_k = dz0*q^k with dz0~U[5,20], q~U[1.0,1.05]; rho0 = rho_s*exp(-z/H) with
    rho_s~U[1.0,1.3], H~U[7000,9000]; S ~ N(0,1) per domain, mean removed.
    """
    rng = np.random.default_rng(seed)
    out = []
    for b in range(ndomains):
        n = int(rng.choice(nxy_choices))
        nz = int(rng.choice(nz_choices))
        dxy = float(rng.choice(BATCH_DXY))
        dz0 = rng.uniform(5.0, 20.0)
        q = rng.uniform(1.0, 1.05)
        rho_s = rng.uniform(1.0, 1.3)
        H = rng.uniform(7000.0, 9000.0)
        sseed = int(rng.integers(0, 2**31 - 1))
        dz = stretched_levels(nz, dz0, q)
        rho = exponential_density(dz, rho_s, H)
        S = normal_source((nz, n, n), sseed) if with_source else None
        out.append(Domain(n, n, nz, dxy, dxy, dz, rho, S, name=f"batch{b}_{n}x{n}x{nz}",
                          extra={"source_seed": sseed}))
    return out


def random_stretched(nx: int, ny: int, nz: int, seed: int, dx: float = 1.0, dy: float = 1.3) -> Domain:
    """Small irregular test problem: random positive dz and rho0, S ~ N(0,1) mean removed."""
    rng = np.random.default_rng(seed)
    dz = rng.uniform(0.5, 2.0, nz)
    rho = rng.uniform(0.6, 1.4, nz)
    S = rng.standard_normal((nz, ny, nx))
    S -= S.mean()
    return Domain(nx, ny, nz, dx, dy, dz, rho, S, name=f"random_{nx}x{ny}x{nz}_s{seed}")


def perturbed_density(nx: int, ny: int, rho0: np.ndarray, eps: float, seed: int, modes: int = 4) -> np.ndarray:
    """rho_ijk = rho0_k (1 + eps g_ijk): a seeded smooth perturbation of a level profile.

    g is a normalised sum of `modes` periodic cosines in x and y (wavenumbers 1..3)
    times a slow variation in z, with max |g| = 1, so rho stays positive for eps < 1.
    Stands in for the horizontally varying density (e.g. moist or terrain-following
    cases) that the FFT solve cannot separate.
    """
    rng = np.random.default_rng(seed)
    rho0 = np.asarray(rho0, dtype=np.float64)
    nz = rho0.size
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    g = np.zeros((nz, ny, nx))
    for _ in range(modes):
        a, b = rng.integers(0, 4, size=2)
        if a == 0 and b == 0:
            a = 1
        ph = rng.uniform(0, 2 * np.pi, size=3)
        g += (np.cos(2 * np.pi * a * i / nx + ph[0]) * np.cos(2 * np.pi * b * j / ny + ph[1])
              * (1.0 + 0.5 * np.cos(np.pi * (k + 0.5) / nz + ph[2])))
    g /= np.abs(g).max()
    return rho0[:, None, None] * (1.0 + eps * g)
